// Double-float 3D FFT convolution for the float64 path's PME (power-of-two
// grids): phi = unnormalised inverse DFT of G(m) * forward DFT(Q).
//
// cuFFT's float64 transforms keep the scarce float64 pipe busy (about 90 us
// for one forward + inverse 64^3 pair on GB300); these passes do the same
// arithmetic in double-float (hi + lo floats, ~48 bits) on the float units.
// Complex transforms of length K along each axis:
//   z forward  (DIF, real float64 or fixed-point input as hi/lo, output bit-reversed)
//   y forward  (DIF)
//   x forward, multiply by G at the bit-reversed frequencies, x inverse (DIT)
//   y inverse  (DIT, bit-reversed input, natural output)
//   z inverse  (DIT), real part written as the hi/lo potential for the gather
// Forward: X(m) = sum_n x(n) exp(-2 pi i m n / K); inverse: exp(+...), no 1/K.
// Each block stages kLines lines of one axis in shared memory (coalesced
// loads: for the y and x passes the kLines lines are neighbours along z), one
// warp transforms one line with radix-2 butterflies between __syncwarp()s.
#include "amp_internal.cuh"

namespace amp {
namespace {

constexpr int kLines = 8;  // lines per block, one warp each

struct cdf {
  dflt re, im;
};

__device__ __forceinline__ cdf c_add(const cdf& a, const cdf& b) { return {df_add(a.re, b.re), df_add(a.im, b.im)}; }
__device__ __forceinline__ cdf c_sub(const cdf& a, const cdf& b) { return {df_sub(a.re, b.re), df_sub(a.im, b.im)}; }
// a * (c - i s)  (forward twiddle)
__device__ __forceinline__ cdf c_mul_fwd(const cdf& a, dflt c, dflt s) {
  return {df_madd(a.im, s, df_mul(a.re, c)), df_sub(df_mul(a.im, c), df_mul(a.re, s))};
}
// a * (c + i s)  (inverse twiddle)
__device__ __forceinline__ cdf c_mul_inv(const cdf& a, dflt c, dflt s) {
  return {df_sub(df_mul(a.re, c), df_mul(a.im, s)), df_madd(a.re, s, df_mul(a.im, c))};
}

__device__ __forceinline__ cdf ld(const float4* p) {
  const float4 v = *p;
  return {{v.x, v.y}, {v.z, v.w}};
}
__device__ __forceinline__ void st(float4* p, const cdf& v) { *p = make_float4(v.re.hi, v.re.lo, v.im.hi, v.im.lo); }

__device__ __forceinline__ int bitrev(int v, int bits) { return (int)(__brev((unsigned)v) >> (32 - bits)); }

// In-place transform of one line x[0..K) in shared memory by the 32 lanes of a warp.
// tw[k] = (cos_hi, cos_lo, sin_hi, sin_lo) of 2 pi k / K, k < K/2.
template <int K, bool kForward>
__device__ __forceinline__ void line_fft(float4* x, const float4* __restrict__ tw) {
  const int lane = threadIdx.x & 31;
  if (kForward) {  // decimation in frequency: natural in, bit-reversed out
    for (int s = K / 2; s >= 1; s >>= 1) {
      for (int b = lane; b < K / 2; b += 32) {
        const int i = (b / s) * 2 * s + (b % s), j = i + s;
        const float4 w = tw[(b % s) * (K / (2 * s))];
        const cdf a = ld(x + i), c = ld(x + j);
        st(x + i, c_add(a, c));
        st(x + j, c_mul_fwd(c_sub(a, c), {w.x, w.y}, {w.z, w.w}));
      }
      __syncwarp();
    }
  } else {  // decimation in time: bit-reversed in, natural out
    for (int s = 1; s <= K / 2; s <<= 1) {
      for (int b = lane; b < K / 2; b += 32) {
        const int i = (b / s) * 2 * s + (b % s), j = i + s;
        const float4 w = tw[(b % s) * (K / (2 * s))];
        const cdf a = ld(x + i), c = c_mul_inv(ld(x + j), {w.x, w.y}, {w.z, w.w});
        st(x + i, c_add(a, c));
        st(x + j, c_sub(a, c));
      }
      __syncwarp();
    }
  }
}

__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }  // -126 <= e <= 127

// A 64-bit fixed-point value v * 2^-s as hi/lo floats: v in three pieces of
// at most 23 bits, each converted exactly, summed error-free.
__device__ __forceinline__ dflt fixed_to_df(long long v, int s) {
  const float a = (float)(int)(v >> 40), b = (float)(int)((v >> 20) & 0xFFFFF), c = (float)(int)(v & 0xFFFFF);
  return df_add(df_two_sum(a * pow2f(40 - s), b * pow2f(20 - s)), dflt{c * pow2f(-s), 0.f});
}

// z forward: lines (x, y) contiguous in the real grid, either float64 or (kFixed)
// 64-bit fixed point scaled by 2^fx_info[0], which is zeroed once read.
template <int K, bool kFixed>
__global__ void __launch_bounds__(32 * kLines) k_fft_z_fwd(const double* __restrict__ q,
                                                          unsigned long long* __restrict__ qfx,
                                                          const int* __restrict__ fx_info, float4* __restrict__ out,
                                                          const float4* __restrict__ tw, const int* __restrict__ stop) {
  if (stop && *stop) return;
  __shared__ float4 sm[kLines][K];
  const long long line0 = (long long)blockIdx.x * kLines;  // line = x*K + y
  // the block's kLines lines are one contiguous run of kLines * K values
  if (kFixed) {
    const int sfx = fx_info[0];
    constexpr int kPer = (kLines * K + 32 * kLines - 1) / (32 * kLines);
    long long v[kPer];
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
      const int e = threadIdx.x + i * 32 * kLines;
      v[i] = e < kLines * K ? (long long)qfx[line0 * K + e] : 0ll;
    }
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
      const int e = threadIdx.x + i * 32 * kLines;
      if (e >= kLines * K) break;
      qfx[line0 * K + e] = 0ull;
      const dflt d = fixed_to_df(v[i], sfx);
      sm[e / K][e % K] = make_float4(d.hi, d.lo, 0.f, 0.f);
    }
  } else {
    for (int e = threadIdx.x; e < kLines * K; e += blockDim.x) {
      const dflt d = df_split(q[line0 * K + e]);
      sm[e / K][e % K] = make_float4(d.hi, d.lo, 0.f, 0.f);
    }
  }
  __syncthreads();
  const int w = threadIdx.x >> 5;
  line_fft<K, true>(sm[w], tw);
  __syncthreads();
  for (int e = threadIdx.x; e < kLines * K; e += blockDim.x) {
    const int l = e / K, k = e % K;
    out[(line0 + l) * K + k] = sm[l][k];
  }
}

// y or x pass over the complex grid g[x][y][z]: lines along axis (1 = y,
// 2 = x), kLines neighbouring z per block. kFusedG: forward, * G, inverse.
template <int K, int kAxis, bool kForward, bool kFusedG>
__global__ void __launch_bounds__(32 * kLines) k_fft_yx(float4* __restrict__ g, const float4* __restrict__ tw,
                                                       const float2* __restrict__ Gdf, const int* __restrict__ stop) {
  if (stop && *stop) return;
  __shared__ float4 sm[kLines][K];
  constexpr int kBits = __builtin_ctz(K);
  // block -> (other index o, z0): o = x for the y pass, y for the x pass
  const int zb = blockIdx.x % (K / kLines), o = blockIdx.x / (K / kLines);
  const int z0 = zb * kLines;
  auto index = [&](int t, int l) -> long long {  // t along the line, l = z offset
    const int z = z0 + l;
    return kAxis == 1 ? ((long long)o * K + t) * K + z : ((long long)t * K + o) * K + z;
  };
  for (int e = threadIdx.x; e < kLines * K; e += blockDim.x) {
    const int t = e / kLines, l = e % kLines;  // consecutive threads: consecutive z
    sm[l][t] = g[index(t, l)];
  }
  __syncthreads();
  const int w = threadIdx.x >> 5;
  if (kFusedG) {
    line_fft<K, true>(sm[w], tw);
    // position t along x holds frequency bitrev(t); y and z are bit-reversed too
    const int lane = threadIdx.x & 31;
    const int my = bitrev(o, kBits), mz = bitrev(z0 + w, kBits);
    for (int t = lane; t < K; t += 32) {
      const float2 gv = Gdf[((long long)bitrev(t, kBits) * K + my) * K + mz];
      const cdf a = ld(&sm[w][t]);
      st(&sm[w][t], {df_mul(a.re, {gv.x, gv.y}), df_mul(a.im, {gv.x, gv.y})});
    }
    __syncwarp();
    line_fft<K, false>(sm[w], tw);
  } else {
    line_fft<K, kForward>(sm[w], tw);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kLines * K; e += blockDim.x) {
    const int t = e / kLines, l = e % kLines;
    g[index(t, l)] = sm[l][t];
  }
}

// z inverse: real part of each point written as hi/lo floats.
template <int K>
__global__ void __launch_bounds__(32 * kLines) k_fft_z_inv(const float4* __restrict__ g, float2* __restrict__ phi,
                                                          const float4* __restrict__ tw, const int* __restrict__ stop) {
  if (stop && *stop) return;
  __shared__ float4 sm[kLines][K];
  const long long line0 = (long long)blockIdx.x * kLines;
  for (int e = threadIdx.x; e < kLines * K; e += blockDim.x) {
    const int l = e / K, k = e % K;
    sm[l][k] = g[(line0 + l) * K + k];
  }
  __syncthreads();
  const int w = threadIdx.x >> 5;
  line_fft<K, false>(sm[w], tw);
  __syncthreads();
  for (int e = threadIdx.x; e < kLines * K; e += blockDim.x) {
    const int l = e / K, k = e % K;
    const float4 v = sm[l][k];
    phi[(line0 + l) * K + k] = make_float2(v.x, v.y);
  }
}

template <int K>
void run_conv(amp_ctx* c, cudaStream_t st, bool fixed) {
  const int lines = K * K;
  const int blocks = lines / kLines;
  const float4* tw = c->fft_tw;
  float4* g = c->fft_grid;
  c->n_launch += 5;
  const int* stop = c->op_stop;
  if (fixed)
    k_fft_z_fwd<K, true><<<blocks, 32 * kLines, 0, st>>>(nullptr, c->gridfx, c->fx_info, g, tw, stop);
  else
    k_fft_z_fwd<K, false><<<blocks, 32 * kLines, 0, st>>>(c->grid64, nullptr, nullptr, g, tw, stop);
  k_fft_yx<K, 1, true, false><<<blocks, 32 * kLines, 0, st>>>(g, tw, nullptr, stop);
  k_fft_yx<K, 2, true, true><<<blocks, 32 * kLines, 0, st>>>(g, tw, c->fft_G, stop);
  k_fft_yx<K, 1, false, false><<<blocks, 32 * kLines, 0, st>>>(g, tw, nullptr, stop);
  k_fft_z_inv<K><<<blocks, 32 * kLines, 0, st>>>(g, c->phi_df, tw, stop);
}

}  // namespace

bool fft_df_supported(int K) { return K == 16 || K == 32 || K == 64 || K == 128; }

// Tables for the double-float FFT: twiddles of length K and the full-spectrum
// influence function as hi/lo pairs (G(mx, my, mz) = G_half at min(mz, K - mz)).
int fft_df_setup(amp_ctx* c, const double* G_half) {
  const int K = c->K;
  const long long ng = (long long)K * K * K;
  int r;
  if (!c->fft_grid) {
    if ((r = dev_alloc(c, &c->fft_grid, ng)) || (r = dev_alloc(c, &c->fft_G, ng)) ||
        (r = dev_alloc(c, &c->fft_tw, K / 2)))
      return r;
  }
  std::vector<float4> tw(K / 2);
  for (int k = 0; k < K / 2; ++k) {
    const double a = 2.0 * M_PI * (double)k / (double)K;
    const double cs = std::cos(a), sn = std::sin(a);
    const float ch = (float)cs, sh = (float)sn;
    tw[k] = make_float4(ch, (float)(cs - (double)ch), sh, (float)(sn - (double)sh));
  }
  std::vector<float2> G(ng);
  const int kh = K / 2 + 1;
  for (int mx = 0; mx < K; ++mx)
    for (int my = 0; my < K; ++my)
      for (int mz = 0; mz < K; ++mz) {
        const int mzh = mz <= K / 2 ? mz : K - mz;
        const double v = G_half[((long long)mx * K + my) * kh + mzh];
        const float h = (float)v;
        G[((long long)mx * K + my) * K + mz] = make_float2(h, (float)(v - (double)h));
      }
  if ((r = cuda_check(c, cudaMemcpyAsync(c->fft_tw, tw.data(), sizeof(float4) * tw.size(), cudaMemcpyHostToDevice,
                                         c->stream),
                      "twiddle upload")) ||
      (r = cuda_check(c, cudaMemcpyAsync(c->fft_G, G.data(), sizeof(float2) * ng, cudaMemcpyHostToDevice, c->stream),
                      "G upload")))
    return r;
  return cuda_check(c, cudaStreamSynchronize(c->stream), "fft tables");
}

// phi (hi/lo floats) = conv(grid) on stream st.
void fft_df_convolve(amp_ctx* c, cudaStream_t st, bool fixed) {
  switch (c->K) {
    case 16: run_conv<16>(c, st, fixed); break;
    case 32: run_conv<32>(c, st, fixed); break;
    case 64: run_conv<64>(c, st, fixed); break;
    case 128: run_conv<128>(c, st, fixed); break;
    default: break;
  }
}

}  // namespace amp
