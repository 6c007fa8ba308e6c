// FP64-accurate apply in double-float arithmetic (placeholder until the kernel lands).
#include "sem_internal.h"

sem_status sem_launch_apply_emu(sem_handle *h, const double *u, double *y, cudaStream_t s) {
  (void)h; (void)u; (void)y; (void)s;
  return sem_fail(SEM_ERR_INVALID, "SEM_FP64_EMU not available yet");
}
