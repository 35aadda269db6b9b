// Double-float 3D FFT convolution for the float64 path's PME (power-of-two
// grids up to 64): phi = unnormalised C2R( G(m) * R2C(Q) ), the same
// transform pair as cuFFT's D2Z / Z2D, with G given on the half spectrum
// mz = 0 .. K/2.
//
// cuFFT's float64 transforms keep the scarce float64 pipe busy (about 90 us
// for one forward + inverse 64^3 pair on GB300); these kernels do the same
// arithmetic in double-float (hi + lo floats, ~48 bits) on the float units,
// in three launches over the half spectrum:
//   A (one cluster of eight CTAs per x plane): two real z lines packed as one complex line
//     (rows y and y + K/2), forward z transforms, the two half spectra
//     separated, then forward y transforms; the plane's half spectrum goes
//     to H[x][mz][my] (my in bit-reversed order);
//   B (lines along x, two neighbouring my per block): forward x transform,
//     times G, inverse x transform, in place;
//   C (one cluster of CTAs per x plane): inverse y transforms, the two real z lines
//     rebuilt from their half spectra as one complex line, inverse z
//     transform; real part -> row y, imaginary part -> row y + K/2 of phi.
// Forward: X(m) = sum_n x(n) exp(-2 pi i m n / K); inverse: exp(+...), no 1/K.
// A warp transforms one line in shared memory with radix-2 butterflies
// between __syncwarp()s (decimation in frequency for the forward transforms,
// natural in / bit-reversed out; decimation in time for the inverse ones).
// Two real lines a, b packed as c = a + i b have spectra
//   A(m) = (C(m) + conj C(K - m)) / 2,  B(m) = (C(m) - conj C(K - m)) / (2i),
// and back, C(m) = A(m) + i B(m) with A(K - m) = conj A(m) (likewise B); the
// imaginary parts of A and B at m = 0 and m = K/2 are dropped, as C2R does.
#include <cooperative_groups.h>

#include "amp_internal.cuh"

namespace amp {
namespace {

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
__device__ __forceinline__ dflt df_half(dflt a) { return {a.hi * 0.5f, a.lo * 0.5f}; }

__device__ __forceinline__ cdf ld(const float4* p) {
  const float4 v = *p;
  return {{v.x, v.y}, {v.z, v.w}};
}
__device__ __forceinline__ void st(float4* p, const cdf& v) { *p = make_float4(v.re.hi, v.re.lo, v.im.hi, v.im.lo); }

__device__ __forceinline__ int bitrev(int v, int bits) { return (int)(__brev((unsigned)v) >> (32 - bits)); }

// In-place transform of one line x[0..K) in shared memory by the 32 lanes of a warp.
// tw[k] = (cos_hi, cos_lo, sin_hi, sin_lo) of 2 pi k / K, k < K/2.
template <int K, bool kForward>
__device__ __forceinline__ void line_fft(float4* x, const float4* tw) {
  const int lane = threadIdx.x & 31;
  if (kForward) {  // decimation in frequency: natural in, bit-reversed out
#pragma unroll
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
#pragma unroll
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

// The plane passes run one cluster of kClus CTAs per x plane: CTA r owns the
// packed rows y' in [r R, (r + 1) R) (R = K / (2 kClus)) for the z
// transforms and the half-spectrum lines mz in [mz_lo(r), mz_lo(r + 1)) for
// the y transforms; the values that cross over are read from the other CTAs'
// shared memory (distributed shared memory) between two cluster barriers.
constexpr int kClus = 8;

template <int K>
struct Plane {
  static constexpr int kH = K / 2 + 1;              // half-spectrum lines
  static constexpr int R = K / 2 / kClus;           // packed rows per CTA
  static constexpr int M = (kH + kClus - 1) / kClus;  // at most this many mz lines per CTA
  static constexpr int kWarps = R > M ? R : M;
  static constexpr int NT = 32 * kWarps;
  static constexpr int kBits = __builtin_ctz(K);
};

__host__ __device__ __forceinline__ int mz_lo(int r, int kH) { return r * kH / kClus; }
__device__ __forceinline__ int mz_owner(int mz, int kH) {
  int r = 0;
  while (r + 1 < kClus && mz_lo(r + 1, kH) <= mz) ++r;
  return r;
}

// Pass A. Input plane x of the real grid, float64 or (kFixed) 64-bit fixed
// point scaled by 2^fx_info[0], which is zeroed once read.
template <int K, bool kFixed>
__global__ void __cluster_dims__(kClus, 1, 1) __launch_bounds__(Plane<K>::NT)
    k_fft_plane_fwd(const double* __restrict__ q, unsigned long long* __restrict__ qfx,
                    const int* __restrict__ fx_info, float4* __restrict__ H, const float4* __restrict__ tw_g,
                    const int* __restrict__ stop) {
  namespace cg = cooperative_groups;
  using PL = Plane<K>;
  constexpr int kH = PL::kH, R = PL::R, NT = PL::NT;
  if (stop && *stop) return;  // the same for every CTA of the cluster
  pdl_wait();
  pdl_trigger();
  __shared__ float4 tw[K / 2];
  __shared__ float4 zl[R][K];        // packed line y' = row y' + i row y' + K/2
  __shared__ float4 Ploc[kH][2 * R]; // separated half spectra of this CTA's rows
  __shared__ float4 yl[PL::M][K];    // this CTA's mz lines over all y
  cg::cluster_group cluster = cg::this_cluster();
  const int r = (int)cluster.block_rank(), x = blockIdx.x / kClus, w = threadIdx.x >> 5;
  const int y0 = r * R;
  for (int k = threadIdx.x; k < K / 2; k += NT) tw[k] = tw_g[k];
  const long long base = (long long)x * K * K;
  const int sfx = kFixed ? fx_info[0] : 0;
  for (int e = threadIdx.x; e < 2 * R * K; e += NT) {
    const int li = e / K % R, half = e / (R * K), z = e % K;
    const long long g = base + (long long)(y0 + li + half * (K / 2)) * K + z;
    const dflt d = kFixed ? fixed_to_df((long long)qfx[g], sfx) : df_split(q[g]);
    float4* p = &zl[li][z];
    if (half == 0) {
      p->x = d.hi;
      p->y = d.lo;
    } else {
      p->z = d.hi;
      p->w = d.lo;
    }
  }
  __syncthreads();
  if (kFixed)  // every value read is in shared memory: zero it for the next spreading
    for (int e = threadIdx.x; e < 2 * R * K; e += NT) {
      const int li = e / K % R, half = e / (R * K), z = e % K;
      qfx[base + (long long)(y0 + li + half * (K / 2)) * K + z] = 0ull;
    }
  if (w < R) line_fft<K, true>(zl[w], tw);
  __syncthreads();
  for (int e = threadIdx.x; e < R * kH; e += NT) {
    const int li = e / kH, mz = e % kH;
    const cdf ck = ld(&zl[li][bitrev(mz & (K - 1), PL::kBits)]);
    const cdf cm = ld(&zl[li][bitrev((K - mz) & (K - 1), PL::kBits)]);
    st(&Ploc[mz][li], {df_half(df_add(ck.re, cm.re)), df_half(df_sub(ck.im, cm.im))});
    st(&Ploc[mz][R + li], {df_half(df_add(ck.im, cm.im)), df_half(df_sub(cm.re, ck.re))});
  }
  cluster.sync();
  const int m0 = mz_lo(r, kH), nm = mz_lo(r + 1, kH) - m0;
  for (int e = threadIdx.x; e < nm * K; e += NT) {
    const int t = e / K, y = e % K;
    const int yp = y % (K / 2), owner = yp / R;
    const float4* src = cluster.map_shared_rank(&Ploc[0][0], owner);
    yl[t][y] = src[(m0 + t) * (2 * R) + (y < K / 2 ? 0 : R) + yp % R];
  }
  cluster.sync();  // no CTA leaves while another still reads its shared memory
  if (w < nm) line_fft<K, true>(yl[w], tw);
  __syncthreads();
  float4* out = H + (long long)x * kH * K;
  for (int e = threadIdx.x; e < nm * K; e += NT) out[(long long)(m0 + e / K) * K + e % K] = yl[e / K][e % K];
}

// Pass B: lines along x of H[x][mz][my], kLinesB neighbouring my per block;
// forward, times G(mx, my, mz), inverse. Position t along x holds
// mx = bitrev(t); position p along y holds my = bitrev(p).
constexpr int kLinesB = 2;
template <int K>
__global__ void __launch_bounds__(32 * kLinesB) k_fft_x_conv(float4* __restrict__ H, const float4* __restrict__ tw_g,
                                                            const float2* __restrict__ Gh,
                                                            const int* __restrict__ stop) {
  if (stop && *stop) return;
  pdl_wait();
  pdl_trigger();
  constexpr int kBits = __builtin_ctz(K), kH = K / 2 + 1;
  constexpr int kGroups = K >= kLinesB ? K / kLinesB : 1;
  __shared__ float4 tw[K / 2];
  __shared__ float4 sm[kLinesB][K];
  const int mz = blockIdx.x / kGroups, p0 = (blockIdx.x % kGroups) * kLinesB;
  for (int k = threadIdx.x; k < K / 2; k += blockDim.x) tw[k] = tw_g[k];
  for (int e = threadIdx.x; e < kLinesB * K; e += blockDim.x) {
    const int t = e / kLinesB, l = e % kLinesB;  // consecutive threads: consecutive my
    sm[l][t] = H[((long long)t * kH + mz) * K + p0 + l];
  }
  __syncthreads();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  line_fft<K, true>(sm[w], tw);
  const int my = bitrev(p0 + w, kBits);
  for (int t = lane; t < K; t += 32) {
    const float2 g = Gh[((long long)bitrev(t, kBits) * K + my) * kH + mz];
    const cdf a = ld(&sm[w][t]);
    st(&sm[w][t], {df_mul(a.re, {g.x, g.y}), df_mul(a.im, {g.x, g.y})});
  }
  __syncwarp();
  line_fft<K, false>(sm[w], tw);
  __syncthreads();
  for (int e = threadIdx.x; e < kLinesB * K; e += blockDim.x) {
    const int t = e / kLinesB, l = e % kLinesB;
    H[((long long)t * kH + mz) * K + p0 + l] = sm[l][t];
  }
}

// Pass C: inverse y transforms of plane x, the real z lines rebuilt pairwise,
// inverse z transforms; phi[x][y][z] as hi/lo floats.
template <int K>
__global__ void __cluster_dims__(kClus, 1, 1) __launch_bounds__(Plane<K>::NT)
    k_fft_plane_inv(const float4* __restrict__ H, float2* __restrict__ phi, const float4* __restrict__ tw_g,
                    const int* __restrict__ stop) {
  namespace cg = cooperative_groups;
  using PL = Plane<K>;
  constexpr int kH = PL::kH, R = PL::R, NT = PL::NT;
  if (stop && *stop) return;
  pdl_wait();
  pdl_trigger();
  __shared__ float4 tw[K / 2];
  __shared__ float4 yl[PL::M][K];  // this CTA's mz lines, then over natural y
  __shared__ float4 zl[R][K];      // packed lines, bit-reversed for the DIT
  cg::cluster_group cluster = cg::this_cluster();
  const int r = (int)cluster.block_rank(), x = blockIdx.x / kClus, w = threadIdx.x >> 5;
  const int y0 = r * R;
  for (int k = threadIdx.x; k < K / 2; k += NT) tw[k] = tw_g[k];
  const int m0 = mz_lo(r, kH), nm = mz_lo(r + 1, kH) - m0;
  const float4* in = H + (long long)x * kH * K;
  for (int e = threadIdx.x; e < nm * K; e += NT) yl[e / K][e % K] = in[(long long)(m0 + e / K) * K + e % K];
  __syncthreads();
  if (w < nm) line_fft<K, false>(yl[w], tw);
  cluster.sync();
  // C(m) = A(m) + i B(m); A = row y', B = row y' + K/2
  for (int e = threadIdx.x; e < R * K; e += NT) {
    const int li = e / K, m = e % K;
    const int mh = m <= K / 2 ? m : K - m;
    const int owner = mz_owner(mh, kH);
    const float4* src = cluster.map_shared_rank(&yl[0][0], owner);
    const int row = (mh - mz_lo(owner, kH)) * K;
    cdf a = ld(&src[row + y0 + li]), b = ld(&src[row + y0 + li + K / 2]);
    if (mh == 0 || mh == K / 2) {
      a.im = {0.f, 0.f};
      b.im = {0.f, 0.f};
    }
    cdf cc;
    if (m <= K / 2)
      cc = {df_sub(a.re, b.im), df_add(a.im, b.re)};
    else
      cc = {df_add(a.re, b.im), df_sub(b.re, a.im)};
    st(&zl[li][bitrev(m, PL::kBits)], cc);
  }
  cluster.sync();  // no CTA leaves while another still reads its shared memory
  if (w < R) line_fft<K, false>(zl[w], tw);
  __syncthreads();
  float2* out = phi + (long long)x * K * K;
  for (int e = threadIdx.x; e < 2 * R * K; e += NT) {
    const int li = e / K % R, half = e / (R * K), z = e % K;
    const float4 v = zl[li][z];
    out[(long long)(y0 + li + half * (K / 2)) * K + z] = half == 0 ? make_float2(v.x, v.y) : make_float2(v.z, v.w);
  }
}

template <int K>
void run_conv(amp_ctx* c, cudaStream_t st, bool fixed) {
  constexpr int kGroups = K >= kLinesB ? K / kLinesB : 1;
  const float4* tw = c->fft_tw;
  float4* H = c->fft_grid;
  const int* stop = c->op_stop;
  c->n_launch += 3;
  const double* qnull = nullptr;
  unsigned long long* fxnull = nullptr;
  const int* infonull = nullptr;
  if (fixed)
    launch_pdl(k_fft_plane_fwd<K, true>, dim3(K * kClus), dim3(Plane<K>::NT), 0, st, qnull, c->gridfx, c->fx_info, H,
               tw, stop);
  else
    launch_pdl(k_fft_plane_fwd<K, false>, dim3(K * kClus), dim3(Plane<K>::NT), 0, st, c->grid64, fxnull, infonull,
               H, tw, stop);
  launch_pdl(k_fft_x_conv<K>, dim3((K / 2 + 1) * kGroups), dim3(32 * kLinesB), 0, st, H, tw, c->fft_G, stop);
  launch_pdl(k_fft_plane_inv<K>, dim3(K * kClus), dim3(Plane<K>::NT), 0, st, H, c->phi_df, tw, stop);
}

}  // namespace

bool fft_df_supported(int K) { return K == 16 || K == 32 || K == 64; }

// Tables for the double-float FFT: twiddles of length K and the influence
// function on the half spectrum as hi/lo pairs, G_half[(mx K + my)(K/2+1) + mz].
int fft_df_setup(amp_ctx* c, const double* G_half) {
  const int K = c->K;
  const long long nh = (long long)K * K * (K / 2 + 1);
  int r;
  if (!c->fft_grid) {
    if ((r = dev_alloc(c, &c->fft_grid, nh)) || (r = dev_alloc(c, &c->fft_G, nh)) ||
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
  std::vector<float2> G(nh);
  for (long long k = 0; k < nh; ++k) {
    const float h = (float)G_half[k];
    G[k] = make_float2(h, (float)(G_half[k] - (double)h));
  }
  if ((r = cuda_check(c, cudaMemcpyAsync(c->fft_tw, tw.data(), sizeof(float4) * tw.size(), cudaMemcpyHostToDevice,
                                         c->stream),
                      "twiddle upload")) ||
      (r = cuda_check(c, cudaMemcpyAsync(c->fft_G, G.data(), sizeof(float2) * nh, cudaMemcpyHostToDevice, c->stream),
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
    default: break;
  }
}

}  // namespace amp
