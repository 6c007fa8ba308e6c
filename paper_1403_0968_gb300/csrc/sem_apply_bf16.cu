// FP32 apply with BF16-stored factors (sem_apply_kernel.cuh, factor type __nv_bfloat16); separate
// translation unit so that it compiles in parallel with the other precisions.
#include "sem_apply_pipe.cuh"

template sem_status dispatch_apply<float, __nv_bfloat16>(const sem_handle *, const float *, float *, const void *,
                                                         const float *, const float *, double *, SemScalars *,
                                                         int *, cudaStream_t);
