// The double-float variant of the own FFT convolution (amp_fft.cuh) on the
// grids above 50 (the smaller ones are in amp_fft_df.cu).
#include "amp_fft.cuh"

namespace amp {

// phi_df = conv(gridfx) on stream st when K is one of the larger grids
// (returns false otherwise); gridfx is zeroed on the way.
bool fft_df_convolve_hi(amp_ctx* c, cudaStream_t st) {
  using namespace fft;
  switch (c->K) {
#define AMP_FFT_CASE(k)                                                                                           \
  case k:                                                                                                         \
    run_conv<k, DfTr>(c, st, c->gridfx, c->fx_info, c->fft_grid, c->fft_tw, c->fft_G, c->phi_df, c->op_stop); \
    return true;
    AMP_FFT_SIZES_HI(AMP_FFT_CASE)
#undef AMP_FFT_CASE
    default:
      return false;
  }
}

}  // namespace amp
