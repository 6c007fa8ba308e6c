// Double-float apply instantiated for n = 2..9 (N = 1..8); see sem_emu.cuh.
#include "sem_emu.cuh"

namespace semu {
template sem_status launch_emu<2>(const sem_handle *h, const double *u, double *y, double *partials, SemScalars *scal, cudaStream_t s);
template sem_status launch_emu<3>(const sem_handle *h, const double *u, double *y, double *partials, SemScalars *scal, cudaStream_t s);
template sem_status launch_emu<4>(const sem_handle *h, const double *u, double *y, double *partials, SemScalars *scal, cudaStream_t s);
template sem_status launch_emu<5>(const sem_handle *h, const double *u, double *y, double *partials, SemScalars *scal, cudaStream_t s);
template sem_status launch_emu<6>(const sem_handle *h, const double *u, double *y, double *partials, SemScalars *scal, cudaStream_t s);
template sem_status launch_emu<7>(const sem_handle *h, const double *u, double *y, double *partials, SemScalars *scal, cudaStream_t s);
template sem_status launch_emu<8>(const sem_handle *h, const double *u, double *y, double *partials, SemScalars *scal, cudaStream_t s);
template sem_status launch_emu<9>(const sem_handle *h, const double *u, double *y, double *partials, SemScalars *scal, cudaStream_t s);
}  // namespace semu
