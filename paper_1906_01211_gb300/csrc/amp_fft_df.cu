// The double-float variant of the own FFT convolution (amp_fft.cuh): the
// float64 path's T*mu and the mixed path's float64 check; grids up to 50
// here, the larger ones in amp_fft_df_hi.cu.
#include "amp_fft.cuh"

namespace amp {

// phi_df (hi/lo floats) = conv(gridfx) on stream st; gridfx is zeroed on the way.
bool fft_df_convolve_hi(amp_ctx* c, cudaStream_t st);

void fft_df_convolve(amp_ctx* c, cudaStream_t st) {
  using namespace fft;
  if (fft_df_convolve_hi(c, st)) return;
  switch (c->K) {
#define AMP_FFT_CASE(k)                                                                                           \
  case k:                                                                                                         \
    run_conv<k, DfTr>(c, st, c->gridfx, c->fx_info, c->fft_grid, c->fft_tw, c->fft_G, c->phi_df, c->op_stop); \
    break;
    AMP_FFT_SIZES_LO(AMP_FFT_CASE)
#undef AMP_FFT_CASE
    default:
      break;
  }
}

}  // namespace amp
