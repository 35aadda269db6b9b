// The float64 variant of the own FFT convolution (amp_fft.cuh): the
// permanent field's reciprocal part, once per geometry.
#include "amp_fft.cuh"

namespace amp {

// phi = conv(grid) on stream st (phi and grid distinct); grid is zeroed on the way.
void fft_f64_convolve(amp_ctx* c, cudaStream_t st, double* grid, double* phi) {
  using namespace fft;
  switch (c->K) {
#define AMP_FFT_CASE(k)                                                                               \
  case k:                                                                                             \
    run_conv<k, F64Tr>(c, st, grid, nullptr, c->fft_grid64, c->fft_tw64, c->G64, phi, nullptr); \
    break;
    AMP_FFT_SIZES(AMP_FFT_CASE)
#undef AMP_FFT_CASE
    default:
      break;
  }
}

}  // namespace amp
