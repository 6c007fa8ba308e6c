// FP64 instantiation of the apply kernel (sem_apply_kernel.cuh); separate translation unit so
// that the precisions compile in parallel.
#include "sem_apply_pipe.cuh"

template sem_status dispatch_apply<double, double>(const sem_handle *, const double *, double *, const void *,
                                           const double *, const double *, double *, SemScalars *, int *,
                                           cudaStream_t);
