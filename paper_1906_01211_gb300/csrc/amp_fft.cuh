// 3D FFT convolution for the PME on even grids K = 2^a 3^b 5^c up to 128:
// phi = unnormalised C2R( G(m) * R2C(Q) ), the same transform pair as cuFFT's
// D2Z / Z2D (R2C / C2R), with G given on the half spectrum mz = 0 .. K/2.
// Three arithmetics share the code:
//   double-float (the float64 path's T*mu and the mixed path's float64
//     check): the grid arrives in 64-bit fixed point; values are hi + lo
//     floats (~48 bits) on the float units, since float64 transforms keep the
//     scarce float64 pipe busy; phi leaves as hi/lo pairs;
//   float32 (the mixed path's operator): float grid in, float phi out;
//   float64 (the permanent field, once per geometry): double grid in,
//     double phi out, on the float64 pipe.
// Three launches over the half spectrum:
//   A (one cluster of kClus CTAs per x plane): two real z lines packed as one
//     complex line (rows y and y + K/2), forward z transforms, the two half
//     spectra separated, then forward y transforms; the plane's half
//     spectrum goes to H[x][mz][my];
//   B (lines along x, two neighbouring my per block): forward x transform,
//     times G, inverse x transform, in place;
//   C (one cluster of CTAs per x plane): inverse y transforms, the two real
//     z lines rebuilt from their half spectra as one complex line, inverse z
//     transform; real part -> row y, imaginary part -> row y + K/2 of phi.
// Forward: X(m) = sum_n x(n) exp(-2 pi i m n / K); inverse: exp(+...), no 1/K.
// A warp transforms one line in shared memory by the Stockham autosort
// algorithm (natural order in and out, a second line buffer per warp), in
// stages of radix 4, 2, 5 or 3 (Govindaraju et al., SC 2008: stage j of
// radix R with Ns the product of the earlier radices reads x[j + r K/R],
// twiddles it by exp(-+2 pi i r (j mod Ns) / (Ns R)), takes an R-point DFT
// and writes it to (j div Ns) Ns R + (j mod Ns) + k Ns). The 3- and 5-point
// DFTs use the symmetric forms with cos and sin of 2 pi/R, read from the
// twiddle table. Two real lines a, b packed as c = a + i b have spectra
//   A(m) = (C(m) + conj C(K - m)) / 2,  B(m) = (C(m) - conj C(K - m)) / (2i),
// and back, C(m) = A(m) + i B(m) with A(K - m) = conj A(m) (likewise B); the
// imaginary parts of A and B at m = 0 and m = K/2 are dropped, as C2R does.
#pragma once

#include <cooperative_groups.h>

#include <mutex>

#include "amp_internal.cuh"

namespace amp {
namespace fft {
namespace {  // one private copy per translation unit

// ---- scalar arithmetic of the three variants (dflt: double-float, float, double)
__device__ __forceinline__ dflt r_add(dflt a, dflt b) { return df_add(a, b); }
__device__ __forceinline__ dflt r_sub(dflt a, dflt b) { return df_sub(a, b); }
__device__ __forceinline__ dflt r_mul(dflt a, dflt b) { return df_mul(a, b); }
__device__ __forceinline__ dflt r_madd(dflt a, dflt b, dflt c) { return df_madd(a, b, c); }
__device__ __forceinline__ dflt r_half(dflt a) { return {a.hi * 0.5f, a.lo * 0.5f}; }
__device__ __forceinline__ dflt r_neg(dflt a) { return df_neg(a); }
__device__ __forceinline__ double r_add(double a, double b) { return a + b; }
__device__ __forceinline__ double r_sub(double a, double b) { return a - b; }
__device__ __forceinline__ double r_mul(double a, double b) { return a * b; }
__device__ __forceinline__ double r_madd(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ double r_half(double a) { return a * 0.5; }
__device__ __forceinline__ double r_neg(double a) { return -a; }
__device__ __forceinline__ float r_add(float a, float b) { return a + b; }
__device__ __forceinline__ float r_sub(float a, float b) { return a - b; }
__device__ __forceinline__ float r_mul(float a, float b) { return a * b; }
__device__ __forceinline__ float r_madd(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ float r_half(float a) { return a * 0.5f; }
__device__ __forceinline__ float r_neg(float a) { return -a; }

template <typename R>
struct Cx {
  R re, im;
};

template <typename R>
__device__ __forceinline__ Cx<R> c_add(const Cx<R>& a, const Cx<R>& b) { return {r_add(a.re, b.re), r_add(a.im, b.im)}; }
template <typename R>
__device__ __forceinline__ Cx<R> c_sub(const Cx<R>& a, const Cx<R>& b) { return {r_sub(a.re, b.re), r_sub(a.im, b.im)}; }
template <typename R>
__device__ __forceinline__ Cx<R> c_scale(const Cx<R>& a, R s) { return {r_mul(a.re, s), r_mul(a.im, s)}; }
// -i a (forward) or +i a (inverse)
template <bool kFwd, typename R>
__device__ __forceinline__ Cx<R> c_rot(const Cx<R>& a) {
  return kFwd ? Cx<R>{a.im, r_neg(a.re)} : Cx<R>{r_neg(a.im), a.re};
}
// a * (c - i s) (forward twiddle) or a * (c + i s) (inverse)
template <typename R>
__device__ __forceinline__ Cx<R> c_mul_fwd(const Cx<R>& a, R c, R s) {
  return {r_madd(a.im, s, r_mul(a.re, c)), r_sub(r_mul(a.im, c), r_mul(a.re, s))};
}
template <typename R>
__device__ __forceinline__ Cx<R> c_mul_inv(const Cx<R>& a, R c, R s) {
  return {r_sub(r_mul(a.re, c), r_mul(a.im, s)), r_madd(a.re, s, r_mul(a.im, c))};
}

// ---- storage of the variants in shared and global memory
// double-float: complex (re hi, re lo, im hi, im lo) as float4, twiddle
// (cos hi, lo, sin hi, lo) as float4, G and phi as (hi, lo) float2;
// float32: complex and twiddle (cos, sin) as float2, G and phi as float;
// float64: complex and twiddle as double2, G and phi as double.
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
__device__ __forceinline__ void st(float4* p, const Cx<dflt>& v) { *p = make_float4(v.re.hi, v.re.lo, v.im.hi, v.im.lo); }
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
__device__ __forceinline__ void set_re(float4* p, dflt v) {
  p->x = v.hi;
  p->y = v.lo;
}
__device__ __forceinline__ void set_im(float4* p, dflt v) {
  p->z = v.hi;
  p->w = v.lo;
}
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

__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }  // -126 <= e <= 127

// A 64-bit fixed-point value v * 2^-s as hi/lo floats: v in three pieces of
// at most 23 bits, each converted exactly, summed error-free.
__device__ __forceinline__ dflt fixed_to_df(long long v, int s) {
  const float a = (float)(int)(v >> 40), b = (float)(int)((v >> 20) & 0xFFFFF), c = (float)(int)(v & 0xFFFFF);
  return df_add(df_two_sum(a * pow2f(40 - s), b * pow2f(20 - s)), dflt{c * pow2f(-s), 0.f});
}
__device__ __forceinline__ dflt grid_in(const unsigned long long* q, long long g, int sfx) {
  return fixed_to_df((long long)q[g], sfx);
}
__device__ __forceinline__ float grid_in(const float* q, long long g, int) { return q[g]; }

// ---- the line transform
// Radix of the stage with m points of the line left to factor: 4, then
// 2, 5, 3. At K = 64 radix-4 stages have 16 butterflies for a warp's 32
// lanes; serialised under ncu the three double-float passes then take 39 us
// against 34.7 us with six radix-2 stages, but inside the solve, beside the
// real-space kernel, the radix-4 passes are the faster ones (same GB300,
// water-23556: float64 solve 0.90 against 0.94 ms, the FFT phase 0.47
// against 0.54 ms per step): fewer stages, fewer shared-memory round trips
// and warp barriers to share the SMs with.
__host__ __device__ constexpr int pick_radix(int m) {
  return m % 4 == 0 ? 4 : (m % 2 == 0 ? 2 : (m % 5 == 0 ? 5 : 3));
}
__host__ __device__ constexpr int n_stages(int m) { return m <= 1 ? 0 : 1 + n_stages(m / pick_radix(m)); }
__host__ __device__ constexpr bool smooth(int m) {
  return m <= 1 ? m == 1 : (m % 2 == 0 ? smooth(m / 2) : (m % 3 == 0 ? smooth(m / 3) : (m % 5 == 0 ? smooth(m / 5) : false)));
}

// the R-point DFT of v in place (R = 2, 3, 4, 5); tw the K-entry table
template <int R, int K, bool kFwd, typename Tr>
__device__ __forceinline__ void dft_small(Cx<typename Tr::R>* v, const typename Tr::T* tw) {
  using Rl = typename Tr::R;
  if constexpr (R == 2) {
    const Cx<Rl> a = v[0], b = v[1];
    v[0] = c_add(a, b);
    v[1] = c_sub(a, b);
  } else if constexpr (R == 4) {
    const Cx<Rl> a = c_add(v[0], v[2]), b = c_sub(v[0], v[2]), c = c_add(v[1], v[3]);
    const Cx<Rl> d = c_rot<kFwd>(c_sub(v[1], v[3]));
    v[0] = c_add(a, c);
    v[1] = c_add(b, d);
    v[2] = c_sub(a, c);
    v[3] = c_sub(b, d);
  } else if constexpr (R == 3) {
    const Rl s3 = tw_sin(tw[K / 3]);  // sin(2 pi / 3)
    const Cx<Rl> t1 = c_add(v[1], v[2]), t2 = c_sub(v[1], v[2]);
    const Cx<Rl> a = c_sub(v[0], Cx<Rl>{r_half(t1.re), r_half(t1.im)});
    const Cx<Rl> b = c_rot<kFwd>(c_scale(t2, s3));
    v[0] = c_add(v[0], t1);
    v[1] = c_add(a, b);
    v[2] = c_sub(a, b);
  } else {  // R == 5
    const Rl c1 = tw_cos(tw[K / 5]), s1 = tw_sin(tw[K / 5]), c2 = tw_cos(tw[2 * K / 5]), s2 = tw_sin(tw[2 * K / 5]);
    const Cx<Rl> t1 = c_add(v[1], v[4]), t2 = c_add(v[2], v[3]), t3 = c_sub(v[1], v[4]), t4 = c_sub(v[2], v[3]);
    const Cx<Rl> a1 = c_add(v[0], c_add(c_scale(t1, c1), c_scale(t2, c2)));
    const Cx<Rl> a2 = c_add(v[0], c_add(c_scale(t1, c2), c_scale(t2, c1)));
    const Cx<Rl> b1 = c_rot<kFwd>(c_add(c_scale(t3, s1), c_scale(t4, s2)));
    const Cx<Rl> b2 = c_rot<kFwd>(c_sub(c_scale(t3, s2), c_scale(t4, s1)));
    v[0] = c_add(v[0], c_add(t1, t2));
    v[1] = c_add(a1, b1);
    v[4] = c_sub(a1, b1);
    v[2] = c_add(a2, b2);
    v[3] = c_sub(a2, b2);
  }
}

// one Stockham stage of radix pick_radix(K / Ns), src -> dst, by one warp
template <int K, int Ns, bool kFwd, typename Tr>
__device__ __forceinline__ void stockham_stage(const typename Tr::S* src, typename Tr::S* dst,
                                               const typename Tr::T* tw) {
  using Rl = typename Tr::R;
  constexpr int R = pick_radix(K / Ns), Q = K / R, step = K / (Ns * R);
  for (int j = threadIdx.x & 31; j < Q; j += 32) {
    const int jm = j % Ns;
    Cx<Rl> v[R];
    v[0] = ld(src + j);
#pragma unroll
    for (int r = 1; r < R; ++r) {
      const typename Tr::T w = tw[r * jm * step];
      const Cx<Rl> a = ld(src + j + r * Q);
      v[r] = kFwd ? c_mul_fwd(a, tw_cos(w), tw_sin(w)) : c_mul_inv(a, tw_cos(w), tw_sin(w));
    }
    dft_small<R, K, kFwd, Tr>(v, tw);
    const int base = (j / Ns) * Ns * R + jm;
#pragma unroll
    for (int k = 0; k < R; ++k) st(dst + base + k * Ns, v[k]);
  }
}

template <int K, int Ns, bool kFwd, typename Tr>
__device__ __forceinline__ void stockham(typename Tr::S* a, typename Tr::S* b, const typename Tr::T* tw) {
  if constexpr (Ns < K) {
    stockham_stage<K, Ns, kFwd, Tr>(a, b, tw);
    __syncwarp();
    stockham<K, Ns * pick_radix(K / Ns), kFwd, Tr>(b, a, tw);
  }
}

// In-place transform of the line x[0..K) in shared memory by the 32 lanes of
// a warp, with the work line w[0..K); tw[k] = cos and sin of 2 pi k / K.
template <int K, bool kFwd, typename Tr>
__device__ __forceinline__ void line_fft(typename Tr::S* x, typename Tr::S* w, const typename Tr::T* tw) {
  stockham<K, 1, kFwd, Tr>(x, w, tw);
  if constexpr (n_stages(K) % 2 == 1) {
    for (int k = threadIdx.x & 31; k < K; k += 32) x[k] = w[k];
    __syncwarp();
  }
}

// ---- the plane passes: one cluster of kClus CTAs per x plane. CTA r owns
// the packed rows y' in [r R, (r + 1) R) (R = K / (2 kClus)) for the z
// transforms and the half-spectrum lines mz in [mz_lo(r), mz_lo(r + 1)) for
// the y transforms; the values that cross over are read from the other CTAs'
// shared memory (distributed shared memory) between two cluster barriers.
// kClus divides K/2 and keeps a CTA at six warps or fewer (max(R, M) <= 6):
// the largest such divisor up to 8, else the smallest one up to 16 (a
// non-portable cluster size, opted into at launch), else the largest divisor
// up to 16. Small CTAs matter in the solve, where the plane passes run
// beside the real-space kernel, which keeps ~49k of an SM's 64k registers:
// a 352-thread CTA of 56 registers does not fit beside it, a 192-thread one
// does. Shared memory is dynamic.
__host__ __device__ constexpr int warps_of(int K, int d) {
  return (K / 2 / d) > ((K / 2 + 1 + d - 1) / d) ? (K / 2 / d) : ((K / 2 + 1 + d - 1) / d);
}
__host__ __device__ constexpr int clus_of(int K) {
  int best = 1;
  for (int d = 1; d <= 8; ++d)
    if ((K / 2) % d == 0 && warps_of(K, d) <= 6) best = d;
  if (warps_of(K, best) <= 6) return best;
  for (int d = 9; d <= 16; ++d)
    if ((K / 2) % d == 0 && warps_of(K, d) <= 6) return d;
  for (int d = 16; d >= 1; --d)
    if ((K / 2) % d == 0) return d;
  return 1;
}

template <int K>
struct Plane {
  static constexpr int kClus = clus_of(K);
  static constexpr int kH = K / 2 + 1;               // half-spectrum lines
  static constexpr int R = K / 2 / kClus;            // packed rows per CTA
  static constexpr int M = (kH + kClus - 1) / kClus;  // at most this many mz lines per CTA
  static constexpr int kWarps = R > M ? R : M;
  static constexpr int NT = 32 * kWarps;
};

__host__ __device__ __forceinline__ int mz_lo(int r, int kH, int kClus) { return r * kH / kClus; }
__device__ __forceinline__ int mz_owner(int mz, int kH, int kClus) {
  int r = 0;
  while (r + 1 < kClus && mz_lo(r + 1, kH, kClus) <= mz) ++r;
  return r;
}

// dynamic shared memory of the plane passes (bytes)
template <int K, typename Tr>
constexpr size_t smem_fwd() {
  using PL = Plane<K>;
  return sizeof(typename Tr::T) * K +
         sizeof(typename Tr::S) * (PL::R * K + PL::kH * 2 * PL::R + PL::M * K + PL::kWarps * K);
}
template <int K, typename Tr>
constexpr size_t smem_inv() {
  using PL = Plane<K>;
  return sizeof(typename Tr::T) * K + sizeof(typename Tr::S) * (PL::M * K + PL::R * K + PL::kWarps * K);
}

// Pass A. Input plane x of the real grid q (64-bit fixed point scaled by
// 2^fx_info[0] in double-float, float in float32, double in float64),
// zeroed once read so that the next spreading starts from zero.
template <int K, typename Tr>
__global__ void __launch_bounds__(Plane<K>::NT)
    k_fft_plane_fwd(typename Tr::In* __restrict__ q, const int* __restrict__ fx_info, typename Tr::S* __restrict__ H,
                    const typename Tr::T* __restrict__ tw_g, const int* __restrict__ stop) {
  namespace cg = cooperative_groups;
  using PL = Plane<K>;
  using Rl = typename Tr::R;
  using S = typename Tr::S;
  using T = typename Tr::T;
  constexpr int kH = PL::kH, R = PL::R, NT = PL::NT, kC = PL::kClus;
  pdl_wait();  // first: a kernel never completes before the one it depends on
  if (stop && *stop) return;  // the same for every CTA of the cluster
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* tw = reinterpret_cast<T*>(smem_raw);
  S* zl = reinterpret_cast<S*>(tw + K);  // [R][K] packed line y' = row y' + i row y' + K/2
  S* Ploc = zl + R * K;                  // [kH][2R] separated half spectra of this CTA's rows
  S* yl = Ploc + kH * 2 * R;             // [M][K] this CTA's mz lines over all y
  S* wk = yl + PL::M * K;                // [kWarps][K] work lines
  cg::cluster_group cluster = cg::this_cluster();
  const int r = (int)cluster.block_rank(), x = blockIdx.x / kC, w = threadIdx.x >> 5;
  const int y0 = r * R;
  for (int k = threadIdx.x; k < K; k += NT) tw[k] = tw_g[k];
  const long long base = (long long)x * K * K;
  const int sfx = fx_info ? fx_info[0] : 0;
  for (int e = threadIdx.x; e < 2 * R * K; e += NT) {
    const int li = e / K % R, half = e / (R * K), z = e % K;
    const long long g = base + (long long)(y0 + li + half * (K / 2)) * K + z;
    const Rl d = grid_in(q, g, sfx);
    if (half == 0)
      set_re(&zl[li * K + z], d);
    else
      set_im(&zl[li * K + z], d);
  }
  __syncthreads();
  // every value read is in shared memory: zero it for the next spreading
  for (int e = threadIdx.x; e < 2 * R * K; e += NT) {
    const int li = e / K % R, half = e / (R * K), z = e % K;
    q[base + (long long)(y0 + li + half * (K / 2)) * K + z] = typename Tr::In(0);
  }
  if (w < R) line_fft<K, true, Tr>(zl + w * K, wk + w * K, tw);
  __syncthreads();
  for (int e = threadIdx.x; e < R * kH; e += NT) {
    const int li = e / kH, mz = e % kH;
    const Cx<Rl> ck = ld(&zl[li * K + mz]);
    const Cx<Rl> cm = ld(&zl[li * K + (K - mz) % K]);
    st(&Ploc[mz * 2 * R + li], Cx<Rl>{r_half(r_add(ck.re, cm.re)), r_half(r_sub(ck.im, cm.im))});
    st(&Ploc[mz * 2 * R + R + li], Cx<Rl>{r_half(r_add(ck.im, cm.im)), r_half(r_sub(cm.re, ck.re))});
  }
  cluster.sync();
  const int m0 = mz_lo(r, kH, kC), nm = mz_lo(r + 1, kH, kC) - m0;
  for (int e = threadIdx.x; e < nm * K; e += NT) {
    const int t = e / K, y = e % K;
    const int yp = y % (K / 2), owner = yp / R;
    const S* src = cluster.map_shared_rank(Ploc, owner);
    yl[t * K + y] = src[(m0 + t) * (2 * R) + (y < K / 2 ? 0 : R) + yp % R];
  }
  cluster.sync();  // no CTA leaves while another still reads its shared memory
  if (w < nm) line_fft<K, true, Tr>(yl + w * K, wk + w * K, tw);
  __syncthreads();
  S* out = H + (long long)x * kH * K;
  for (int e = threadIdx.x; e < nm * K; e += NT) out[(long long)(m0 + e / K) * K + e % K] = yl[e];
}

// Pass B: lines along x of H[x][mz][my], kLinesB neighbouring my per block;
// forward, times G(mx, my, mz), inverse.
constexpr int kLinesB = 2;
template <int K, typename Tr>
__global__ void __launch_bounds__(32 * kLinesB) k_fft_x_conv(typename Tr::S* __restrict__ H,
                                                            const typename Tr::T* __restrict__ tw_g,
                                                            const typename Tr::G* __restrict__ Gh,
                                                            const int* __restrict__ stop) {
  using Rl = typename Tr::R;
  pdl_wait();  // first: a kernel never completes before the one it depends on
  if (stop && *stop) return;
  pdl_trigger();
  constexpr int kH = K / 2 + 1, kGroups = K / kLinesB;
  __shared__ typename Tr::T tw[K];
  __shared__ typename Tr::S sm[kLinesB][K];
  __shared__ typename Tr::S wk[kLinesB][K];
  const int mz = blockIdx.x / kGroups, p0 = (blockIdx.x % kGroups) * kLinesB;
  for (int k = threadIdx.x; k < K; k += blockDim.x) tw[k] = tw_g[k];
  for (int e = threadIdx.x; e < kLinesB * K; e += blockDim.x) {
    const int t = e / kLinesB, l = e % kLinesB;  // consecutive threads: consecutive my
    sm[l][t] = H[((long long)t * kH + mz) * K + p0 + l];
  }
  __syncthreads();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  line_fft<K, true, Tr>(sm[w], wk[w], tw);
  const int my = p0 + w;
  for (int t = lane; t < K; t += 32) {
    const Rl g = g_val(Gh[((long long)t * K + my) * kH + mz]);
    const Cx<Rl> a = ld(&sm[w][t]);
    st(&sm[w][t], Cx<Rl>{r_mul(a.re, g), r_mul(a.im, g)});
  }
  __syncwarp();
  line_fft<K, false, Tr>(sm[w], wk[w], tw);
  __syncthreads();
  for (int e = threadIdx.x; e < kLinesB * K; e += blockDim.x) {
    const int t = e / kLinesB, l = e % kLinesB;
    H[((long long)t * kH + mz) * K + p0 + l] = sm[l][t];
  }
}

// Pass C: inverse y transforms of plane x, the real z lines rebuilt pairwise,
// inverse z transforms; phi[x][y][z].
template <int K, typename Tr>
__global__ void __launch_bounds__(Plane<K>::NT)
    k_fft_plane_inv(const typename Tr::S* __restrict__ H, typename Tr::P* __restrict__ phi,
                    const typename Tr::T* __restrict__ tw_g, const int* __restrict__ stop) {
  namespace cg = cooperative_groups;
  using PL = Plane<K>;
  using Rl = typename Tr::R;
  using S = typename Tr::S;
  using T = typename Tr::T;
  constexpr int kH = PL::kH, R = PL::R, NT = PL::NT, kC = PL::kClus;
  pdl_wait();  // first: a kernel never completes before the one it depends on
  if (stop && *stop) return;
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* tw = reinterpret_cast<T*>(smem_raw);
  S* yl = reinterpret_cast<S*>(tw + K);  // [M][K] this CTA's mz lines over y
  S* zl = yl + PL::M * K;                // [R][K] packed lines
  S* wk = zl + R * K;                    // [kWarps][K] work lines
  cg::cluster_group cluster = cg::this_cluster();
  const int r = (int)cluster.block_rank(), x = blockIdx.x / kC, w = threadIdx.x >> 5;
  const int y0 = r * R;
  for (int k = threadIdx.x; k < K; k += NT) tw[k] = tw_g[k];
  const int m0 = mz_lo(r, kH, kC), nm = mz_lo(r + 1, kH, kC) - m0;
  const S* in = H + (long long)x * kH * K;
  for (int e = threadIdx.x; e < nm * K; e += NT) yl[e] = in[(long long)(m0 + e / K) * K + e % K];
  __syncthreads();
  if (w < nm) line_fft<K, false, Tr>(yl + w * K, wk + w * K, tw);
  cluster.sync();
  // C(m) = A(m) + i B(m); A = row y', B = row y' + K/2
  for (int e = threadIdx.x; e < R * K; e += NT) {
    const int li = e / K, m = e % K;
    const int mh = m <= K / 2 ? m : K - m;
    const int owner = mz_owner(mh, kH, kC);
    const S* src = cluster.map_shared_rank(yl, owner);
    const int row = (mh - mz_lo(owner, kH, kC)) * K;
    Cx<Rl> a = ld(&src[row + y0 + li]), b = ld(&src[row + y0 + li + K / 2]);
    if (mh == 0 || mh == K / 2) {
      a.im = r_zero<Rl>();
      b.im = r_zero<Rl>();
    }
    Cx<Rl> cc;
    if (m <= K / 2)
      cc = {r_sub(a.re, b.im), r_add(a.im, b.re)};
    else
      cc = {r_add(a.re, b.im), r_sub(b.re, a.im)};
    st(&zl[li * K + m], cc);
  }
  cluster.sync();  // no CTA leaves while another still reads its shared memory
  if (w < R) line_fft<K, false, Tr>(zl + w * K, wk + w * K, tw);
  __syncthreads();
  typename Tr::P* out = phi + (long long)x * K * K;
  for (int e = threadIdx.x; e < 2 * R * K; e += NT) {
    const int li = e / K % R, half = e / (R * K), z = e % K;
    const S v = zl[li * K + z];
    out[(long long)(y0 + li + half * (K / 2)) * K + z] = half == 0 ? re_out(v) : im_out(v);
  }
}

// A plane pass: clusters of kClus CTAs along x, programmatic dependent
// launch as launch_pdl.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_plane(void (*kernel)(KArgs...), int clus, dim3 grid, dim3 block, size_t smem,
                                cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  attr[1].id = cudaLaunchAttributeClusterDimension;
  attr[1].val.clusterDim.x = (unsigned)clus;
  attr[1].val.clusterDim.y = 1;
  attr[1].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// The three passes on stream st (the opt-ins to more than 48 KB of dynamic
// shared memory and to clusters above 8 CTAs are made once per
// instantiation).
template <int K, typename Tr>
void run_conv(amp_ctx* c, cudaStream_t st, typename Tr::In* grid, const int* fx_info, typename Tr::S* H,
              const typename Tr::T* tw, const typename Tr::G* G, typename Tr::P* phi, const int* stop) {
  static_assert(K % 2 == 0 && smooth(K), "even 2^a 3^b 5^c grids only");
  constexpr int kGroups = K / kLinesB, kC = Plane<K>::kClus;
  constexpr size_t sa = smem_fwd<K, Tr>(), sc = smem_inv<K, Tr>();
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute(k_fft_plane_fwd<K, Tr>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sa);
    cudaFuncSetAttribute(k_fft_plane_inv<K, Tr>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sc);
    if (kC > 8) {
      cudaFuncSetAttribute(k_fft_plane_fwd<K, Tr>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      cudaFuncSetAttribute(k_fft_plane_inv<K, Tr>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    }
  });
  c->n_launch += 3;
  launch_plane(k_fft_plane_fwd<K, Tr>, kC, dim3(K * kC), dim3(Plane<K>::NT), sa, st, grid, fx_info, H, tw, stop);
  launch_pdl(k_fft_x_conv<K, Tr>, dim3((K / 2 + 1) * kGroups), dim3(32 * kLinesB), 0, st, H, tw, G, stop);
  launch_plane(k_fft_plane_inv<K, Tr>, kC, dim3(K * kC), dim3(Plane<K>::NT), sc, st, H, phi, tw, stop);
}

// The supported grid sizes (even, 2^a 3^b 5^c, 16 .. 128; the others use
// cuFFT), for the dispatch;
// the double-float variant is compiled in two halves (build time).
#define AMP_FFT_SIZES_LO(X) X(16) X(18) X(20) X(24) X(30) X(32) X(36) X(40) X(48) X(50)
#define AMP_FFT_SIZES_HI(X) X(60) X(64) X(72) X(80) X(96) X(100) X(120) X(128)
#define AMP_FFT_SIZES(X) AMP_FFT_SIZES_LO(X) AMP_FFT_SIZES_HI(X)

}  // namespace
}  // namespace fft
}  // namespace amp
