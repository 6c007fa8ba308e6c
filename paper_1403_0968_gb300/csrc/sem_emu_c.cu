// Double-float apply instantiated for n = 14..16 (N = 13..15); see sem_emu.cuh.
#include "sem_emu.cuh"

namespace semu {
template sem_status launch_emu<14>(const sem_handle *h, const double *u, double *y, double *partials, SemScalars *scal, cudaStream_t s);
template sem_status launch_emu<15>(const sem_handle *h, const double *u, double *y, double *partials, SemScalars *scal, cudaStream_t s);
template sem_status launch_emu<16>(const sem_handle *h, const double *u, double *y, double *partials, SemScalars *scal, cudaStream_t s);
}  // namespace semu
