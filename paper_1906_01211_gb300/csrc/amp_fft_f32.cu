// The float32 variant of the own FFT convolution (amp_fft.cuh): the mixed
// path's operator.
#include "amp_fft.cuh"

namespace amp {

// phi32 = conv(spread32) on stream st; spread32 is zeroed on the way.
void fft_f32_convolve(amp_ctx* c, cudaStream_t st) {
  using namespace fft;
  switch (c->K) {
#define AMP_FFT_CASE(k)                                                                                                \
  case k:                                                                                                              \
    run_conv<k, F32Tr>(c, st, c->spread32, nullptr, c->fft_grid32, c->fft_tw32, c->G32, c->phi32, c->op_stop); \
    break;
    AMP_FFT_SIZES(AMP_FFT_CASE)
#undef AMP_FFT_CASE
    default:
      break;
  }
}

}  // namespace amp
