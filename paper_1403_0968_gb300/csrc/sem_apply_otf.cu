// FP32 apply with the geometric factors recomputed at every node from the element's trilinear map
// (sem_apply_kernel.cuh, OtfGeo); separate translation unit so that it compiles in parallel.
#include "sem_apply_pipe.cuh"

template sem_status dispatch_apply<float, OtfGeo>(const sem_handle *, const float *, float *, const void *,
                                                  const float *, const float *, double *, SemScalars *, int *,
                                                  cudaStream_t);
template sem_status dispatch_apply_batch<float, OtfGeo>(int, const BatchEntry *, int, int64_t, int64_t, const float *,
                                                        float *, const float *, const double *, const double *,
                                                        double *, int, cudaStream_t);
