// FP32 instantiation of the apply kernel (sem_apply_kernel.cuh); separate translation unit so
// that the precisions compile in parallel.
#include "sem_apply_pipe.cuh"

template sem_status dispatch_apply<float, float>(const sem_handle *, const float *, float *, const void *, const float *,
                                          const float *, double *, SemScalars *, int *, cudaStream_t);
template sem_status dispatch_apply_batch<float, float>(int, const BatchEntry *, int, int64_t, int64_t, const float *,
                                                       float *, const float *, const double *, const double *,
                                                       double *, int, cudaStream_t);
