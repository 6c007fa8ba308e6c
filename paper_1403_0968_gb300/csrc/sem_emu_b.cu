// Double-float apply instantiated for n = 10..13 (N = 9..12); see sem_emu.cuh.
#include "sem_emu.cuh"

namespace semu {
template sem_status launch_emu<10>(const sem_handle *h, const double *u, double *y, double *partials, SemScalars *scal, cudaStream_t s);
template sem_status launch_emu<11>(const sem_handle *h, const double *u, double *y, double *partials, SemScalars *scal, cudaStream_t s);
template sem_status launch_emu<12>(const sem_handle *h, const double *u, double *y, double *partials, SemScalars *scal, cudaStream_t s);
template sem_status launch_emu<13>(const sem_handle *h, const double *u, double *y, double *partials, SemScalars *scal, cudaStream_t s);
}  // namespace semu
