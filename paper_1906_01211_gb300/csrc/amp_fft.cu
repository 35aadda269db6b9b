// Tables and buffers of the own FFT convolution (amp_fft.cuh; the three
// arithmetics are instantiated in amp_fft_df.cu, amp_fft_f32.cu and
// amp_fft_f64.cu).
#include <cmath>
#include <vector>

#include "amp_fft.cuh"

namespace amp {

bool fft_own_supported(int K) {
  switch (K) {
#define AMP_FFT_CASE(k) case k:
    AMP_FFT_SIZES(AMP_FFT_CASE)
#undef AMP_FFT_CASE
    return true;
    default:
      return false;
  }
}

// Buffers and twiddles of the own FFT (they depend on K only): the half
// spectra of the variants, the influence function's hi/lo split for the
// double-float one (filled by the influence kernel with the float64 and
// float32 copies, which the other two variants read), and the twiddles
// cos, sin of 2 pi k/K, k < K, as hi/lo pairs, floats and doubles. The
// mixed path's float32 variant is set up for K <= kOwnF32MaxK only: on
// larger grids its plane passes (clusters of CTAs of up to 352 threads)
// slow the real-space kernel that runs beside them more than cuFFT's float32
// transforms do (water-96000, K = 100: mixed solve 2.34 ms with the own
// transforms, 1.96 ms with cuFFT; at K = 64 the own ones are faster).
int fft_own_setup(amp_ctx* c) {
  const int K = c->K;
  const long long nh = (long long)K * K * (K / 2 + 1);
  const bool f32 = c->cfg.precision == AMP_MIXED && K <= kOwnF32MaxK;
  int r;
  if (!c->fft_grid) {
    if ((r = dev_alloc(c, &c->fft_grid, nh)) || (r = dev_alloc(c, &c->fft_G, nh)) ||
        (r = dev_alloc(c, &c->fft_tw, K)) || (r = dev_alloc(c, &c->fft_grid64, nh)) ||
        (r = dev_alloc(c, &c->fft_tw64, K)))
      return r;
    if (f32 && ((r = dev_alloc(c, &c->fft_grid32, nh)) || (r = dev_alloc(c, &c->fft_tw32, K)))) return r;
  }
  std::vector<float4> tw(K);
  std::vector<float2> tw32(K);
  std::vector<double2> tw64(K);
  for (int k = 0; k < K; ++k) {
    const double a = 2.0 * M_PI * (double)k / (double)K;
    const double cs = std::cos(a), sn = std::sin(a);
    const float ch = (float)cs, sh = (float)sn;
    tw[k] = make_float4(ch, (float)(cs - (double)ch), sh, (float)(sn - (double)sh));
    tw32[k] = make_float2(ch, sh);
    tw64[k] = make_double2(cs, sn);
  }
  if ((r = cuda_check(c, cudaMemcpyAsync(c->fft_tw, tw.data(), sizeof(float4) * tw.size(), cudaMemcpyHostToDevice,
                                         c->stream),
                      "twiddle upload")) ||
      (r = cuda_check(c, cudaMemcpyAsync(c->fft_tw64, tw64.data(), sizeof(double2) * tw64.size(),
                                         cudaMemcpyHostToDevice, c->stream),
                      "twiddle upload")))
    return r;
  if (f32 && (r = cuda_check(c, cudaMemcpyAsync(c->fft_tw32, tw32.data(), sizeof(float2) * tw32.size(),
                                                 cudaMemcpyHostToDevice, c->stream),
                             "twiddle upload")))
    return r;
  return cuda_check(c, cudaStreamSynchronize(c->stream), "fft tables");
}

}  // namespace amp
