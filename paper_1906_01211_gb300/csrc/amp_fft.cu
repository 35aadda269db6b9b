// 3D FFT convolution for the PME of power-of-two grids up to 64:
// phi = unnormalised C2R( G(m) * R2C(Q) ), the same transform pair as cuFFT's
// D2Z / Z2D (R2C / C2R), with G given on the half spectrum mz = 0 .. K/2.
// Two arithmetics share the code:
//   double-float (the float64 path and the mixed path's float64 check): the
//     grid arrives in 64-bit fixed point; values are hi + lo floats (~48
//     bits) on the float units, since cuFFT's float64 transforms keep the
//     scarce float64 pipe busy (about 90 us for one forward + inverse 64^3
//     pair on GB300); phi leaves as hi/lo pairs;
//   float32 (the mixed path's operator): float grid in, float phi out;
//   float64 (the permanent field, once per geometry): double grid in,
//     double phi out, on the float64 pipe.
// Three launches over the half spectrum:
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

// ---- scalar arithmetic of the two variants (dflt: double-float, float)
__device__ __forceinline__ dflt r_add(dflt a, dflt b) { return df_add(a, b); }
__device__ __forceinline__ dflt r_sub(dflt a, dflt b) { return df_sub(a, b); }
__device__ __forceinline__ dflt r_mul(dflt a, dflt b) { return df_mul(a, b); }
__device__ __forceinline__ dflt r_madd(dflt a, dflt b, dflt c) { return df_madd(a, b, c); }
__device__ __forceinline__ dflt r_half(dflt a) { return {a.hi * 0.5f, a.lo * 0.5f}; }
__device__ __forceinline__ double r_add(double a, double b) { return a + b; }
__device__ __forceinline__ double r_sub(double a, double b) { return a - b; }
__device__ __forceinline__ double r_mul(double a, double b) { return a * b; }
__device__ __forceinline__ double r_madd(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ double r_half(double a) { return a * 0.5; }
__device__ __forceinline__ float r_add(float a, float b) { return a + b; }
__device__ __forceinline__ float r_sub(float a, float b) { return a - b; }
__device__ __forceinline__ float r_mul(float a, float b) { return a * b; }
__device__ __forceinline__ float r_madd(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ float r_half(float a) { return a * 0.5f; }

template <typename R>
struct Cx {
  R re, im;
};

template <typename R>
__device__ __forceinline__ Cx<R> c_add(const Cx<R>& a, const Cx<R>& b) { return {r_add(a.re, b.re), r_add(a.im, b.im)}; }
template <typename R>
__device__ __forceinline__ Cx<R> c_sub(const Cx<R>& a, const Cx<R>& b) { return {r_sub(a.re, b.re), r_sub(a.im, b.im)}; }
// a * (c - i s)  (forward twiddle)
template <typename R>
__device__ __forceinline__ Cx<R> c_mul_fwd(const Cx<R>& a, R c, R s) {
  return {r_madd(a.im, s, r_mul(a.re, c)), r_sub(r_mul(a.im, c), r_mul(a.re, s))};
}
// a * (c + i s)  (inverse twiddle)
template <typename R>
__device__ __forceinline__ Cx<R> c_mul_inv(const Cx<R>& a, R c, R s) {
  return {r_sub(r_mul(a.re, c), r_mul(a.im, s)), r_madd(a.re, s, r_mul(a.im, c))};
}

// ---- storage of the two variants in shared and global memory
// double-float: complex (re hi, re lo, im hi, im lo) as float4, twiddle
// (cos hi, lo, sin hi, lo) as float4, G and phi as (hi, lo) float2;
// float32: complex and twiddle (cos, sin) as float2, G and phi as float.
struct DfTr {
  using R = dflt;
  using S = float4;
  using T = float4;
  using G = float2;
  using P = float2;
  using In = unsigned long long;  // 64-bit fixed-point grid
};
struct F32Tr {
  using R = float;
  using S = float2;
  using T = float2;
  using G = float;
  using P = float;
  using In = float;
};
// float64: complex and twiddle (cos, sin) as double2, G and phi as double
struct F64Tr {
  using R = double;
  using S = double2;
  using T = double2;
  using G = double;
  using P = double;
  using In = double;
};

__device__ __forceinline__ Cx<dflt> ld(const float4* p) {
  const float4 v = *p;
  return {{v.x, v.y}, {v.z, v.w}};
}
__device__ __forceinline__ void st(float4* p, const Cx<dflt>& v) {
  *p = make_float4(v.re.hi, v.re.lo, v.im.hi, v.im.lo);
}
__device__ __forceinline__ Cx<float> ld(const float2* p) {
  const float2 v = *p;
  return {v.x, v.y};
}
__device__ __forceinline__ void st(float2* p, const Cx<float>& v) { *p = make_float2(v.re, v.im); }
__device__ __forceinline__ Cx<double> ld(const double2* p) {
  const double2 v = *p;
  return {v.x, v.y};
}
__device__ __forceinline__ void st(double2* p, const Cx<double>& v) { *p = make_double2(v.re, v.im); }
__device__ __forceinline__ void set_re(double2* p, double v) { p->x = v; }
__device__ __forceinline__ void set_im(double2* p, double v) { p->y = v; }
__device__ __forceinline__ double re_out(const double2& v) { return v.x; }
__device__ __forceinline__ double im_out(const double2& v) { return v.y; }
__device__ __forceinline__ double tw_cos(const double2& w) { return w.x; }
__device__ __forceinline__ double tw_sin(const double2& w) { return w.y; }
__device__ __forceinline__ double g_val(double g) { return g; }
__device__ __forceinline__ double grid_in(const double* q, long long g, int) { return q[g]; }
__device__ __forceinline__ void set_re(float4* p, dflt v) { p->x = v.hi; p->y = v.lo; }
__device__ __forceinline__ void set_im(float4* p, dflt v) { p->z = v.hi; p->w = v.lo; }
__device__ __forceinline__ void set_re(float2* p, float v) { p->x = v; }
__device__ __forceinline__ void set_im(float2* p, float v) { p->y = v; }
__device__ __forceinline__ float2 re_out(const float4& v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 im_out(const float4& v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float re_out(const float2& v) { return v.x; }
__device__ __forceinline__ float im_out(const float2& v) { return v.y; }
__device__ __forceinline__ dflt tw_cos(const float4& w) { return {w.x, w.y}; }
__device__ __forceinline__ dflt tw_sin(const float4& w) { return {w.z, w.w}; }
__device__ __forceinline__ float tw_cos(const float2& w) { return w.x; }
__device__ __forceinline__ float tw_sin(const float2& w) { return w.y; }
__device__ __forceinline__ dflt g_val(const float2& g) { return {g.x, g.y}; }
__device__ __forceinline__ float g_val(float g) { return g; }
template <typename R>
__device__ __forceinline__ R r_zero();
template <>
__device__ __forceinline__ dflt r_zero<dflt>() { return {0.f, 0.f}; }
template <>
__device__ __forceinline__ float r_zero<float>() { return 0.f; }
template <>
__device__ __forceinline__ double r_zero<double>() { return 0.0; }

__device__ __forceinline__ int bitrev(int v, int bits) { return (int)(__brev((unsigned)v) >> (32 - bits)); }

// In-place transform of one line x[0..K) in shared memory by the 32 lanes of
// a warp; tw[k] = cos and sin of 2 pi k / K, k < K/2.
template <int K, bool kForward, typename Tr>
__device__ __forceinline__ void line_fft(typename Tr::S* x, const typename Tr::T* tw) {
  using R = typename Tr::R;
  const int lane = threadIdx.x & 31;
  if (kForward) {  // decimation in frequency: natural in, bit-reversed out
#pragma unroll
    for (int s = K / 2; s >= 1; s >>= 1) {
      for (int b = lane; b < K / 2; b += 32) {
        const int i = (b / s) * 2 * s + (b % s), j = i + s;
        const typename Tr::T w = tw[(b % s) * (K / (2 * s))];
        const Cx<R> a = ld(x + i), c = ld(x + j);
        st(x + i, c_add(a, c));
        st(x + j, c_mul_fwd(c_sub(a, c), tw_cos(w), tw_sin(w)));
      }
      __syncwarp();
    }
  } else {  // decimation in time: bit-reversed in, natural out
#pragma unroll
    for (int s = 1; s <= K / 2; s <<= 1) {
      for (int b = lane; b < K / 2; b += 32) {
        const int i = (b / s) * 2 * s + (b % s), j = i + s;
        const typename Tr::T w = tw[(b % s) * (K / (2 * s))];
        const Cx<R> a = ld(x + i), c = c_mul_inv(ld(x + j), tw_cos(w), tw_sin(w));
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
// grid value in the variant's arithmetic
__device__ __forceinline__ dflt grid_in(const unsigned long long* q, long long g, int sfx) {
  return fixed_to_df((long long)q[g], sfx);
}
__device__ __forceinline__ float grid_in(const float* q, long long g, int) { return q[g]; }

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

// Pass A. Input plane x of the real grid q (64-bit fixed point scaled by
// 2^fx_info[0] in double-float, float in float32), zeroed once read so that
// the next spreading starts from zero.
template <int K, typename Tr>
__global__ void __cluster_dims__(kClus, 1, 1) __launch_bounds__(Plane<K>::NT)
    k_fft_plane_fwd(typename Tr::In* __restrict__ q, const int* __restrict__ fx_info, typename Tr::S* __restrict__ H,
                    const typename Tr::T* __restrict__ tw_g, const int* __restrict__ stop) {
  namespace cg = cooperative_groups;
  using PL = Plane<K>;
  using R_ = typename Tr::R;
  using S = typename Tr::S;
  constexpr int kH = PL::kH, R = PL::R, NT = PL::NT;
  if (stop && *stop) return;  // the same for every CTA of the cluster
  pdl_wait();
  pdl_trigger();
  __shared__ typename Tr::T tw[K / 2];
  __shared__ S zl[R][K];        // packed line y' = row y' + i row y' + K/2
  __shared__ S Ploc[kH][2 * R]; // separated half spectra of this CTA's rows
  __shared__ S yl[PL::M][K];    // this CTA's mz lines over all y
  cg::cluster_group cluster = cg::this_cluster();
  const int r = (int)cluster.block_rank(), x = blockIdx.x / kClus, w = threadIdx.x >> 5;
  const int y0 = r * R;
  for (int k = threadIdx.x; k < K / 2; k += NT) tw[k] = tw_g[k];
  const long long base = (long long)x * K * K;
  const int sfx = fx_info ? fx_info[0] : 0;
  for (int e = threadIdx.x; e < 2 * R * K; e += NT) {
    const int li = e / K % R, half = e / (R * K), z = e % K;
    const long long g = base + (long long)(y0 + li + half * (K / 2)) * K + z;
    const R_ d = grid_in(q, g, sfx);
    if (half == 0)
      set_re(&zl[li][z], d);
    else
      set_im(&zl[li][z], d);
  }
  __syncthreads();
  // every value read is in shared memory: zero it for the next spreading
  for (int e = threadIdx.x; e < 2 * R * K; e += NT) {
    const int li = e / K % R, half = e / (R * K), z = e % K;
    q[base + (long long)(y0 + li + half * (K / 2)) * K + z] = typename Tr::In(0);
  }
  if (w < R) line_fft<K, true, Tr>(zl[w], tw);
  __syncthreads();
  for (int e = threadIdx.x; e < R * kH; e += NT) {
    const int li = e / kH, mz = e % kH;
    const Cx<R_> ck = ld(&zl[li][bitrev(mz & (K - 1), PL::kBits)]);
    const Cx<R_> cm = ld(&zl[li][bitrev((K - mz) & (K - 1), PL::kBits)]);
    st(&Ploc[mz][li], Cx<R_>{r_half(r_add(ck.re, cm.re)), r_half(r_sub(ck.im, cm.im))});
    st(&Ploc[mz][R + li], Cx<R_>{r_half(r_add(ck.im, cm.im)), r_half(r_sub(cm.re, ck.re))});
  }
  cluster.sync();
  const int m0 = mz_lo(r, kH), nm = mz_lo(r + 1, kH) - m0;
  for (int e = threadIdx.x; e < nm * K; e += NT) {
    const int t = e / K, y = e % K;
    const int yp = y % (K / 2), owner = yp / R;
    const S* src = cluster.map_shared_rank(&Ploc[0][0], owner);
    yl[t][y] = src[(m0 + t) * (2 * R) + (y < K / 2 ? 0 : R) + yp % R];
  }
  cluster.sync();  // no CTA leaves while another still reads its shared memory
  if (w < nm) line_fft<K, true, Tr>(yl[w], tw);
  __syncthreads();
  S* out = H + (long long)x * kH * K;
  for (int e = threadIdx.x; e < nm * K; e += NT) out[(long long)(m0 + e / K) * K + e % K] = yl[e / K][e % K];
}

// Pass B: lines along x of H[x][mz][my], kLinesB neighbouring my per block;
// forward, times G(mx, my, mz), inverse. Position t along x holds
// mx = bitrev(t); position p along y holds my = bitrev(p).
constexpr int kLinesB = 2;
template <int K, typename Tr>
__global__ void __launch_bounds__(32 * kLinesB) k_fft_x_conv(typename Tr::S* __restrict__ H,
                                                            const typename Tr::T* __restrict__ tw_g,
                                                            const typename Tr::G* __restrict__ Gh,
                                                            const int* __restrict__ stop) {
  using R_ = typename Tr::R;
  if (stop && *stop) return;
  pdl_wait();
  pdl_trigger();
  constexpr int kBits = __builtin_ctz(K), kH = K / 2 + 1;
  constexpr int kGroups = K >= kLinesB ? K / kLinesB : 1;
  __shared__ typename Tr::T tw[K / 2];
  __shared__ typename Tr::S sm[kLinesB][K];
  const int mz = blockIdx.x / kGroups, p0 = (blockIdx.x % kGroups) * kLinesB;
  for (int k = threadIdx.x; k < K / 2; k += blockDim.x) tw[k] = tw_g[k];
  for (int e = threadIdx.x; e < kLinesB * K; e += blockDim.x) {
    const int t = e / kLinesB, l = e % kLinesB;  // consecutive threads: consecutive my
    sm[l][t] = H[((long long)t * kH + mz) * K + p0 + l];
  }
  __syncthreads();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  line_fft<K, true, Tr>(sm[w], tw);
  const int my = bitrev(p0 + w, kBits);
  for (int t = lane; t < K; t += 32) {
    const R_ g = g_val(Gh[((long long)bitrev(t, kBits) * K + my) * kH + mz]);
    const Cx<R_> a = ld(&sm[w][t]);
    st(&sm[w][t], Cx<R_>{r_mul(a.re, g), r_mul(a.im, g)});
  }
  __syncwarp();
  line_fft<K, false, Tr>(sm[w], tw);
  __syncthreads();
  for (int e = threadIdx.x; e < kLinesB * K; e += blockDim.x) {
    const int t = e / kLinesB, l = e % kLinesB;
    H[((long long)t * kH + mz) * K + p0 + l] = sm[l][t];
  }
}

// Pass C: inverse y transforms of plane x, the real z lines rebuilt pairwise,
// inverse z transforms; phi[x][y][z].
template <int K, typename Tr>
__global__ void __cluster_dims__(kClus, 1, 1) __launch_bounds__(Plane<K>::NT)
    k_fft_plane_inv(const typename Tr::S* __restrict__ H, typename Tr::P* __restrict__ phi,
                    const typename Tr::T* __restrict__ tw_g, const int* __restrict__ stop) {
  namespace cg = cooperative_groups;
  using PL = Plane<K>;
  using R_ = typename Tr::R;
  using S = typename Tr::S;
  constexpr int kH = PL::kH, R = PL::R, NT = PL::NT;
  if (stop && *stop) return;
  pdl_wait();
  pdl_trigger();
  __shared__ typename Tr::T tw[K / 2];
  __shared__ S yl[PL::M][K];  // this CTA's mz lines, then over natural y
  __shared__ S zl[R][K];      // packed lines, bit-reversed for the DIT
  cg::cluster_group cluster = cg::this_cluster();
  const int r = (int)cluster.block_rank(), x = blockIdx.x / kClus, w = threadIdx.x >> 5;
  const int y0 = r * R;
  for (int k = threadIdx.x; k < K / 2; k += NT) tw[k] = tw_g[k];
  const int m0 = mz_lo(r, kH), nm = mz_lo(r + 1, kH) - m0;
  const S* in = H + (long long)x * kH * K;
  for (int e = threadIdx.x; e < nm * K; e += NT) yl[e / K][e % K] = in[(long long)(m0 + e / K) * K + e % K];
  __syncthreads();
  if (w < nm) line_fft<K, false, Tr>(yl[w], tw);
  cluster.sync();
  // C(m) = A(m) + i B(m); A = row y', B = row y' + K/2
  for (int e = threadIdx.x; e < R * K; e += NT) {
    const int li = e / K, m = e % K;
    const int mh = m <= K / 2 ? m : K - m;
    const int owner = mz_owner(mh, kH);
    const S* src = cluster.map_shared_rank(&yl[0][0], owner);
    const int row = (mh - mz_lo(owner, kH)) * K;
    Cx<R_> a = ld(&src[row + y0 + li]), b = ld(&src[row + y0 + li + K / 2]);
    if (mh == 0 || mh == K / 2) {
      a.im = r_zero<R_>();
      b.im = r_zero<R_>();
    }
    Cx<R_> cc;
    if (m <= K / 2)
      cc = {r_sub(a.re, b.im), r_add(a.im, b.re)};
    else
      cc = {r_add(a.re, b.im), r_sub(b.re, a.im)};
    st(&zl[li][bitrev(m, PL::kBits)], cc);
  }
  cluster.sync();  // no CTA leaves while another still reads its shared memory
  if (w < R) line_fft<K, false, Tr>(zl[w], tw);
  __syncthreads();
  typename Tr::P* out = phi + (long long)x * K * K;
  for (int e = threadIdx.x; e < 2 * R * K; e += NT) {
    const int li = e / K % R, half = e / (R * K), z = e % K;
    const S v = zl[li][z];
    out[(long long)(y0 + li + half * (K / 2)) * K + z] = half == 0 ? re_out(v) : im_out(v);
  }
}

template <int K, typename Tr>
void run_conv(amp_ctx* c, cudaStream_t st, typename Tr::In* grid, const int* fx_info, typename Tr::S* H,
              const typename Tr::T* tw, const typename Tr::G* G, typename Tr::P* phi) {
  constexpr int kGroups = K >= kLinesB ? K / kLinesB : 1;
  const int* stop = c->op_stop;
  c->n_launch += 3;
  launch_pdl(k_fft_plane_fwd<K, Tr>, dim3(K * kClus), dim3(Plane<K>::NT), 0, st, grid, fx_info, H, tw, stop);
  launch_pdl(k_fft_x_conv<K, Tr>, dim3((K / 2 + 1) * kGroups), dim3(32 * kLinesB), 0, st, H, tw, G, stop);
  launch_pdl(k_fft_plane_inv<K, Tr>, dim3(K * kClus), dim3(Plane<K>::NT), 0, st, H, phi, tw, stop);
}

}  // namespace

bool fft_own_supported(int K) { return K == 16 || K == 32 || K == 64; }

// Buffers and twiddles of the own FFT (they depend on K only): the half
// spectra of the three variants, the influence function's hi/lo split for the
// double-float one (filled by the influence kernel with the float64 and
// float32 copies, which the other two variants read), and the twiddles
// cos, sin of 2 pi k/K as hi/lo pairs, floats and doubles.
int fft_own_setup(amp_ctx* c) {
  const int K = c->K;
  const long long nh = (long long)K * K * (K / 2 + 1);
  const bool f32 = c->cfg.precision == AMP_MIXED;
  int r;
  if (!c->fft_grid) {
    if ((r = dev_alloc(c, &c->fft_grid, nh)) || (r = dev_alloc(c, &c->fft_G, nh)) ||
        (r = dev_alloc(c, &c->fft_tw, K / 2)) || (r = dev_alloc(c, &c->fft_grid64, nh)) ||
        (r = dev_alloc(c, &c->fft_tw64, K / 2)))
      return r;
    if (f32 && ((r = dev_alloc(c, &c->fft_grid32, nh)) || (r = dev_alloc(c, &c->fft_tw32, K / 2)))) return r;
  }
  std::vector<float4> tw(K / 2);
  std::vector<float2> tw32(K / 2);
  std::vector<double2> tw64(K / 2);
  for (int k = 0; k < K / 2; ++k) {
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

// phi_df (hi/lo floats) = conv(gridfx) in double-float on stream st; gridfx
// is zeroed on the way.
void fft_df_convolve(amp_ctx* c, cudaStream_t st) {
  switch (c->K) {
    case 16: run_conv<16, DfTr>(c, st, c->gridfx, c->fx_info, c->fft_grid, c->fft_tw, c->fft_G, c->phi_df); break;
    case 32: run_conv<32, DfTr>(c, st, c->gridfx, c->fx_info, c->fft_grid, c->fft_tw, c->fft_G, c->phi_df); break;
    case 64: run_conv<64, DfTr>(c, st, c->gridfx, c->fx_info, c->fft_grid, c->fft_tw, c->fft_G, c->phi_df); break;
    default: break;
  }
}

// phi = conv(grid) in float64 on stream st (phi and grid distinct); grid is
// zeroed on the way.
void fft_f64_convolve(amp_ctx* c, cudaStream_t st, double* grid, double* phi) {
  const int* none = nullptr;
  const int* stop = c->op_stop;
  c->op_stop = nullptr;
  switch (c->K) {
    case 16: run_conv<16, F64Tr>(c, st, grid, none, c->fft_grid64, c->fft_tw64, c->G64, phi); break;
    case 32: run_conv<32, F64Tr>(c, st, grid, none, c->fft_grid64, c->fft_tw64, c->G64, phi); break;
    case 64: run_conv<64, F64Tr>(c, st, grid, none, c->fft_grid64, c->fft_tw64, c->G64, phi); break;
    default: break;
  }
  c->op_stop = stop;
}

// phi32 = conv(spread32) in float32 on stream st; spread32 is zeroed on the way.
void fft_f32_convolve(amp_ctx* c, cudaStream_t st) {
  const int* none = nullptr;
  switch (c->K) {
    case 16: run_conv<16, F32Tr>(c, st, c->spread32, none, c->fft_grid32, c->fft_tw32, c->G32, c->phi32); break;
    case 32: run_conv<32, F32Tr>(c, st, c->spread32, none, c->fft_grid32, c->fft_tw32, c->G32, c->phi32); break;
    case 64: run_conv<64, F32Tr>(c, st, c->spread32, none, c->fft_grid32, c->fft_tw32, c->G32, c->phi32); break;
    default: break;
  }
}

}  // namespace amp
