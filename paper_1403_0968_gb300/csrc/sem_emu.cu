// Dispatch of the FP64-accurate double-float apply by order (kernel and launcher: sem_emu.cuh,
// instantiated in sem_emu_a.cu, sem_emu_b.cu, sem_emu_c.cu).
#include "sem_emu.cuh"

namespace semu {
extern template sem_status launch_emu<2>(const sem_handle *h, const double *u, double *y, double *partials, SemScalars *scal, cudaStream_t s);
extern template sem_status launch_emu<3>(const sem_handle *h, const double *u, double *y, double *partials, SemScalars *scal, cudaStream_t s);
extern template sem_status launch_emu<4>(const sem_handle *h, const double *u, double *y, double *partials, SemScalars *scal, cudaStream_t s);
extern template sem_status launch_emu<5>(const sem_handle *h, const double *u, double *y, double *partials, SemScalars *scal, cudaStream_t s);
extern template sem_status launch_emu<6>(const sem_handle *h, const double *u, double *y, double *partials, SemScalars *scal, cudaStream_t s);
extern template sem_status launch_emu<7>(const sem_handle *h, const double *u, double *y, double *partials, SemScalars *scal, cudaStream_t s);
extern template sem_status launch_emu<8>(const sem_handle *h, const double *u, double *y, double *partials, SemScalars *scal, cudaStream_t s);
extern template sem_status launch_emu<9>(const sem_handle *h, const double *u, double *y, double *partials, SemScalars *scal, cudaStream_t s);
extern template sem_status launch_emu<10>(const sem_handle *h, const double *u, double *y, double *partials, SemScalars *scal, cudaStream_t s);
extern template sem_status launch_emu<11>(const sem_handle *h, const double *u, double *y, double *partials, SemScalars *scal, cudaStream_t s);
extern template sem_status launch_emu<12>(const sem_handle *h, const double *u, double *y, double *partials, SemScalars *scal, cudaStream_t s);
extern template sem_status launch_emu<13>(const sem_handle *h, const double *u, double *y, double *partials, SemScalars *scal, cudaStream_t s);
extern template sem_status launch_emu<14>(const sem_handle *h, const double *u, double *y, double *partials, SemScalars *scal, cudaStream_t s);
extern template sem_status launch_emu<15>(const sem_handle *h, const double *u, double *y, double *partials, SemScalars *scal, cudaStream_t s);
extern template sem_status launch_emu<16>(const sem_handle *h, const double *u, double *y, double *partials, SemScalars *scal, cudaStream_t s);
}  // namespace semu

sem_status sem_launch_apply_emu(sem_handle *h, const double *u, double *y, double *partials, cudaStream_t s) {
  // order 7, variant 5: the D-contractions on the tensor cores (measured slower than the
  // CUDA-core kernel on GB300, so never the automatic choice)
  if (h->N == 7 && h->apply_variant == 5) return sem_launch_apply_emu_tc(h, u, y, partials, s);
  SemScalars *scal = h->scal;  // timeouts are recorded there; with partials it also carries the CG step
  switch (h->N) {
#define CASE(NN) \
  case NN:       \
    return semu::launch_emu<NN + 1>(h, u, y, partials, scal, s);
    CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8) CASE(9) CASE(10) CASE(11) CASE(12) CASE(13)
    CASE(14) CASE(15)
#undef CASE
    default:
      return sem_fail(SEM_ERR_INVALID, "order out of range");
  }
}
