// Smooth particle-mesh Ewald (kernels c and c').
//
// Reciprocal-space part of the permanent field and of T*mu (the paper's
// "reciprocal polarization", Section "Sequential performance"; not vectorized
// in the CPU code, Section "Conclusion"). Smooth PME (Essmann et al. 1995)
// with multipolar spreading (Sagui, Pedersen & Darden 2004), order 5:
//   u = K x / L (mod K) per axis, k0 = floor(u), f = u - k0; grid point
//   k0 - t (mod K), t = 0..4, has weight M5(f + t) (cardinal B-spline);
//   Q(g) = sum_i (q_i + d_i . grad + 1/3 Theta_i : grad grad) W_i(g), grad = (K/L) d/du;
//   phi = unnormalised C2R( G . R2C(Q) ),
//   G(m) = exp(-pi^2 m~^2/beta^2) / (pi V m~^2) |b1 b2 b3|^2, G(0) = 0;
//   E_i = -sum_g grad W_i(g) phi(g).
// The permanent multipoles (once per geometry) are spread, transformed and
// gathered in float64 (float64 atomics, cuFFT float64). The dipoles of every
// T*mu (the mixed path's are its float32 operator input) are spread in
// double-float into a 64-bit fixed-point grid, transformed by the
// double-float FFT of amp_fft.cuh on even 2,3,5-smooth grids up to 128 (else
// cuFFT float64, a library call, and a split) and gathered in double-float. The force kernels'
// potentials use float64 (float32 in the mixed path) atomics and cuFFT.
// |b(m)|^2 = 1/|sum_{k=0}^{3} M5(k+1) e^{2 pi i m k/K}|^2; where that sum
// vanishes (m = K/2, even K) the mean of the neighbours m-1, m+1 is used.
#include <cmath>
#include <vector>

#include "amp_internal.cuh"

namespace amp {
namespace {

constexpr int kTh = 3 * 4 * kOrder;    // per atom: 3 axes x derivatives 0..3 x 5 points
constexpr int kThDf = 3 * 2 * kOrder;  // per atom: 3 axes x derivatives 0..1 x 5 points (hi/lo)

// Weights M5(f + t) and their first three derivatives (t = 0..4) by the
// B-spline recursion M_n(u) = [u M_{n-1}(u) + (n - u) M_{n-1}(u - 1)]/(n - 1).
__device__ __forceinline__ void bspline5(double f, double s, double w[4][kOrder]) {
  double m2[2] = {f, 1.0 - f};
  double m3[3], m4[4], m5[5];
  for (int t = 0; t < 3; ++t) {
    const double a = t < 2 ? m2[t] : 0.0, b = t >= 1 ? m2[t - 1] : 0.0;
    m3[t] = ((f + t) * a + (3.0 - f - t) * b) * 0.5;
  }
  for (int t = 0; t < 4; ++t) {
    const double a = t < 3 ? m3[t] : 0.0, b = t >= 1 ? m3[t - 1] : 0.0;
    m4[t] = ((f + t) * a + (4.0 - f - t) * b) * (1.0 / 3.0);
  }
  for (int t = 0; t < 5; ++t) {
    const double a = t < 4 ? m4[t] : 0.0, b = t >= 1 ? m4[t - 1] : 0.0;
    m5[t] = ((f + t) * a + (5.0 - f - t) * b) * 0.25;
  }
  for (int t = 0; t < 5; ++t) {
    const double a4 = t < 4 ? m4[t] : 0.0, b4 = t >= 1 ? m4[t - 1] : 0.0;
    const double a3 = t < 3 ? m3[t] : 0.0, b3 = (t >= 1 && t - 1 < 3) ? m3[t - 1] : 0.0,
                 c3 = (t >= 2 && t - 2 < 3) ? m3[t - 2] : 0.0;
    const double a2 = t < 2 ? m2[t] : 0.0, b2 = (t >= 1 && t - 1 < 2) ? m2[t - 1] : 0.0,
                 c2 = (t >= 2 && t - 2 < 2) ? m2[t - 2] : 0.0, d2 = (t >= 3 && t - 3 < 2) ? m2[t - 3] : 0.0;
    w[0][t] = m5[t];
    w[1][t] = (a4 - b4) * s;
    w[2][t] = (a3 - 2.0 * b3 + c3) * s * s;
    w[3][t] = (a2 - 3.0 * b2 + 3.0 * c2 - d2) * s * s * s;
  }
}

// Float64 B-spline weights (derivatives 0..3, which the force kernels need),
// with their float32 copy when theta32 is given (mixed path); one thread per
// (atom, axis). The base indices are the same as those of k_theta_df (same
// float64 operations).
__global__ void k_theta(int n, const double4_32a* __restrict__ A, double L, int K, double* __restrict__ theta,
                        float* __restrict__ theta32) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 3LL * n) return;
  const int s = (int)(t / 3), ax = (int)(t - 3LL * s);
  const double4_32a a = A[s];
  const double sc = (double)K / L;
  double u = (ax == 0 ? a.x : (ax == 1 ? a.y : a.z)) * sc;
  u = u - (double)K * floor(u * (1.0 / (double)K));
  if (u >= (double)K) u -= (double)K;
  if (u < 0.0) u += (double)K;
  const double k0 = floor(u);
  double w[4][kOrder];
  bspline5(u - k0, sc, w);
  double* th = theta + (long long)kTh * s;
  for (int d = 0; d < 4; ++d)
    for (int k = 0; k < kOrder; ++k) {
      th[(ax * 4 + d) * kOrder + k] = w[d][k];
      if (theta32) theta32[(long long)kTh * s + (ax * 4 + d) * kOrder + k] = (float)w[d][k];
    }
}

// The weights of bspline5 (derivatives 0 and 1) in double-float, from f as
// hi/lo floats and s = K/L: the same recursion (Essmann et al. 1995, Eq.
// 4.1-4.4), about 48 significant bits, on the float units.
__device__ __forceinline__ dflt df_scale(dflt a, float c) { return {a.hi * c, a.lo * c}; }  // c a power of two

__device__ __forceinline__ void bspline5_df(dflt f, dflt s, dflt w[2][kOrder]) {
  const dflt one = {1.f, 0.f}, third = {0.333333343f, -9.93410776e-09f};  // 1/3 = hi + lo
  dflt m2[2] = {f, df_sub(one, f)};
  dflt m3[3], m4[4], m5[5];
  for (int t = 0; t < 3; ++t) {  // M3(f + t) = ((f + t) M2(f + t) + (3 - f - t) M2(f + t - 1)) / 2
    const dflt ft = df_add(f, {(float)t, 0.f}), gt = df_sub({3.f - (float)t, 0.f}, f);
    dflt v = {0.f, 0.f};
    if (t < 2) v = df_mul(ft, m2[t]);
    if (t >= 1) v = df_madd(gt, m2[t - 1], v);
    m3[t] = df_scale(v, 0.5f);
  }
  for (int t = 0; t < 4; ++t) {
    const dflt ft = df_add(f, {(float)t, 0.f}), gt = df_sub({4.f - (float)t, 0.f}, f);
    dflt v = {0.f, 0.f};
    if (t < 3) v = df_mul(ft, m3[t]);
    if (t >= 1) v = df_madd(gt, m3[t - 1], v);
    m4[t] = df_mul(v, third);
  }
  for (int t = 0; t < 5; ++t) {
    const dflt ft = df_add(f, {(float)t, 0.f}), gt = df_sub({5.f - (float)t, 0.f}, f);
    dflt v = {0.f, 0.f};
    if (t < 4) v = df_mul(ft, m4[t]);
    if (t >= 1) v = df_madd(gt, m4[t - 1], v);
    m5[t] = df_scale(v, 0.25f);
  }
  for (int t = 0; t < 5; ++t) {
    const dflt a4 = t < 4 ? m4[t] : dflt{0.f, 0.f}, b4 = t >= 1 ? m4[t - 1] : dflt{0.f, 0.f};
    w[0][t] = m5[t];
    w[1][t] = df_mul(df_sub(a4, b4), s);
  }
}

// One group of four lanes per atom: lane ax < 3 builds axis ax's weights and
// first derivatives in double-float (theta_df) and its base index, which lane
// 0 stores, counting the atom in kcount; fx_info[1] = the largest count (the
// atoms that reach one grid point, for the fixed-point dipole spreading).
__global__ void __launch_bounds__(128) k_theta_df(int n, const double4_32a* __restrict__ A, double L, int K,
                                                   float2 s_df, float2* __restrict__ theta_df,
                                                   int4* __restrict__ gbase, int* __restrict__ kcount,
                                                   int* __restrict__ fx_info) {
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  const int s = gid >> 2, lane4 = gid & 3;
  const bool valid = s < n;
  int base = 0;
  if (valid && lane4 < 3) {
    const double4_32a a = A[s];
    const double x = lane4 == 0 ? a.x : (lane4 == 1 ? a.y : a.z);
    const double sc = (double)K / L;
    double u = x * sc;
    u = u - (double)K * floor(u * (1.0 / (double)K));  // the two tests below fix an off-by-one wrap
    if (u >= (double)K) u -= (double)K;
    if (u < 0.0) u += (double)K;
    const double k0 = floor(u);
    base = (int)k0;
    dflt w[2][kOrder];
    bspline5_df(df_split(u - k0), {s_df.x, s_df.y}, w);
    float2* o = theta_df + (long long)kThDf * s + lane4 * 2 * kOrder;
    for (int t = 0; t < kOrder; ++t) {
      o[t] = make_float2(w[0][t].hi, w[0][t].lo);
      o[kOrder + t] = make_float2(w[1][t].hi, w[1][t].lo);
    }
  }
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int by = __shfl_sync(full, base, lane + 1), bz = __shfl_sync(full, base, lane + 2);
  int cnt = 0;
  if (valid && lane4 == 0) {
    gbase[s] = make_int4(base, by, bz, 0);
    cnt = atomicAdd(kcount + ((long long)base * K + by) * K + bz, 1) + 1;
  }
  // the block's maximum first: one atomic per block, skipped when the stored
  // value is already as large (it only grows)
  __shared__ int wmax[128 / 32];
  const int mc = __reduce_max_sync(full, cnt);
  if (lane == 0) wmax[threadIdx.x >> 5] = mc;
  __syncthreads();
  if (threadIdx.x == 0) {
    int m = 0;
    for (int w = 0; w < 128 / 32; ++w) m = max(m, wmax[w]);
    int* dst = fx_info + 1;
    if (m > __ldcg(dst)) atomicMax(dst, m);
  }
}

template <typename R>
struct Wts {
  R x[3][kOrder], y[3][kOrder], z[3][kOrder];
};

template <typename R>
__device__ __forceinline__ void load_wts(const R* __restrict__ th, int nd, Wts<R>& w) {
  for (int d = 0; d < nd; ++d)
    for (int t = 0; t < kOrder; ++t) {
      w.x[d][t] = th[(0 * 4 + d) * kOrder + t];
      w.y[d][t] = th[(1 * 4 + d) * kOrder + t];
      w.z[d][t] = th[(2 * 4 + d) * kOrder + t];
    }
}

__device__ __forceinline__ int wrapk(int g, int K) { return g < 0 ? g + K : g; }

// Spreading and gathering run one atom per group of kPmeGroup lanes, lane t
// (t < 5) owning the grid plane k0x - t: five times the parallelism of one
// thread per atom, which the float64 pipe needs to stay busy.
constexpr int kPmeGroup = 8;

template <typename R>
__global__ void __launch_bounds__(128) k_spread_multipoles(int n, const R* __restrict__ theta,
                                                           const int4* __restrict__ gbase,
                                                           const double4_32a* __restrict__ A,
                                                           const double4_32a* __restrict__ B,
                                                           const double4_32a* __restrict__ C,
                                                           const double4_32a* __restrict__ D, int K,
                                                           R* __restrict__ grid) {
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  const int s = gid / kPmeGroup, tx = gid % kPmeGroup;
  if (s >= n || tx >= kOrder) return;
  const R* th = theta + (long long)kTh * s;
  R wx[3], wy[3][kOrder], wz[3][kOrder];
  for (int d = 0; d < 3; ++d) {
    wx[d] = th[(0 * 4 + d) * kOrder + tx];
    for (int t = 0; t < kOrder; ++t) {
      wy[d][t] = th[(1 * 4 + d) * kOrder + t];
      wz[d][t] = th[(2 * 4 + d) * kOrder + t];
    }
  }
  const int4 b = gbase[s];
  const double4_32a a = A[s], bb = B[s], c = C[s], d = D[s];
  const R q = (R)a.w, dx = (R)bb.x, dy = (R)bb.y, dz = (R)bb.z;
  const R qxx = (R)c.x, qyy = (R)c.y, qzz = (R)c.z, qxy = (R)c.w, qxz = (R)d.x, qyz = (R)d.y;
  const R third = (R)(1.0 / 3.0), two3 = (R)(2.0 / 3.0);
  const int gx = wrapk(b.x - tx, K);
  for (int ty = 0; ty < kOrder; ++ty) {
    const int gy = wrapk(b.y - ty, K);
    const R x0y0 = wx[0] * wy[0][ty], x1y0 = wx[1] * wy[0][ty], x0y1 = wx[0] * wy[1][ty];
    const R a0 = q * x0y0 + dx * x1y0 + dy * x0y1 +
                 third * (qxx * wx[2] * wy[0][ty] + qyy * wx[0] * wy[2][ty] + (R)2 * qxy * wx[1] * wy[1][ty]);
    const R a1 = dz * x0y0 + two3 * (qxz * x1y0 + qyz * x0y1);
    const R a2 = third * qzz * x0y0;
    R* row = grid + ((long long)gx * K + gy) * K;
    for (int tz = 0; tz < kOrder; ++tz) {
      const int gz = wrapk(b.z - tz, K);
      atomicAdd(row + gz, a0 * wz[0][tz] + a1 * wz[1][tz] + a2 * wz[2][tz]);
    }
  }
}

// The permanent multipoles into the float64 grid (the right-hand side's
// reciprocal part), one thread per (atom, y row, z point), which adds the
// atom's values at the five x planes, P0 w_x + P1 w'_x + P2 w''_x with
//   P0 = q w_y w_z + dy w'_y w_z + dz w_y w'_z + (Qyy w''_y w_z + Qzz w_y w''_z + 2 Qyz w'_y w'_z) / 3,
//   P1 = dx w_y w_z + 2 (Qxy w'_y w_z + Qxz w_y w'_z) / 3,   P2 = Qxx w_y w_z / 3
// (Sagui, Pedersen and Darden 2004, the quadrupole with the 1/3 of the
// traceless form). Every lane works (a float64 instruction holds the float64
// pipe as long for one active lane as for 32).
__global__ void __launch_bounds__(256) k_spread_multipoles64(int n, const double* __restrict__ theta,
                                                             const int4* __restrict__ gbase,
                                                             const double4_32a* __restrict__ A,
                                                             const double4_32a* __restrict__ B,
                                                             const double4_32a* __restrict__ C,
                                                             const double4_32a* __restrict__ D, int K,
                                                             double* __restrict__ grid) {
  const long long item = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (item >= (long long)n * (kOrder * kOrder)) return;
  const int s = (int)(item / (kOrder * kOrder)), tyz = (int)(item - (long long)s * (kOrder * kOrder));
  const int ty = tyz / kOrder, tz = tyz - ty * kOrder;
  const double* th = theta + (long long)kTh * s;
  const double y0 = th[(1 * 4 + 0) * kOrder + ty], y1 = th[(1 * 4 + 1) * kOrder + ty], y2 = th[(1 * 4 + 2) * kOrder + ty];
  const double z0 = th[(2 * 4 + 0) * kOrder + tz], z1 = th[(2 * 4 + 1) * kOrder + tz], z2 = th[(2 * 4 + 2) * kOrder + tz];
  const double4_32a a = A[s], b = B[s], c = C[s], d = D[s];
  const double y0z0 = y0 * z0, y1z0 = y1 * z0, y0z1 = y0 * z1;
  const double P0 = a.w * y0z0 + b.y * y1z0 + b.z * y0z1 +
                    (1.0 / 3.0) * (c.y * y2 * z0 + c.z * y0 * z2 + 2.0 * d.y * y1 * z1);
  const double P1 = b.x * y0z0 + (2.0 / 3.0) * (c.w * y1z0 + d.x * y0z1);
  const double P2 = (1.0 / 3.0) * c.x * y0z0;
  const int4 g = gbase[s];
  double* col = grid + (long long)wrapk(g.y - ty, K) * K + wrapk(g.z - tz, K);
  const long long plane = (long long)K * K;
#pragma unroll
  for (int tx = 0; tx < kOrder; ++tx) {
    const double x0 = th[(0 * 4 + 0) * kOrder + tx], x1 = th[(0 * 4 + 1) * kOrder + tx],
                 x2 = th[(0 * 4 + 2) * kOrder + tx];
    atomicAdd(col + wrapk(g.x - tx, K) * plane, fma(P2, x2, fma(P1, x1, P0 * x0)));
  }
}

template <typename R, typename V>
__global__ void __launch_bounds__(128) k_spread_dipoles(int n, const R* __restrict__ theta,
                                                        const int4* __restrict__ gbase, const V* __restrict__ v,
                                                        int K, R* __restrict__ grid,
                                                        const int* __restrict__ stop = nullptr) {
  if (stop && *stop) return;
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  const int s = gid / kPmeGroup, tx = gid % kPmeGroup;
  if (s >= n || tx >= kOrder) return;
  const R* th = theta + (long long)kTh * s;
  const R wx0 = th[(0 * 4 + 0) * kOrder + tx], wx1 = th[(0 * 4 + 1) * kOrder + tx];
  R wy0[kOrder], wy1[kOrder], wz0[kOrder], wz1[kOrder];
  for (int t = 0; t < kOrder; ++t) {
    wy0[t] = th[(1 * 4 + 0) * kOrder + t];
    wy1[t] = th[(1 * 4 + 1) * kOrder + t];
    wz0[t] = th[(2 * 4 + 0) * kOrder + t];
    wz1[t] = th[(2 * 4 + 1) * kOrder + t];
  }
  const int4 b = gbase[s];
  const V m = v[s];
  const R mx = (R)m.x, my = (R)m.y, mz = (R)m.z;
  const R cx0 = mx * wx1, cx1 = my * wx0, cz = mz * wx0;
  const int gx = wrapk(b.x - tx, K);
  for (int ty = 0; ty < kOrder; ++ty) {
    const int gy = wrapk(b.y - ty, K);
    const R a0 = cx0 * wy0[ty] + cx1 * wy1[ty];
    const R a1 = cz * wy0[ty];
    R* row = grid + ((long long)gx * K + gy) * K;
    for (int tz = 0; tz < kOrder; ++tz) {
      const int gz = wrapk(b.z - tz, K);
      atomicAdd(row + gz, a0 * wz0[tz] + a1 * wz1[tz]);
    }
  }
}

// ---- float64 path: dipoles spread in double-float, accumulated in 64-bit fixed point.
// Integer atomics are exact, so the grid does not depend on the order in which
// atoms arrive, and nothing of the spreading runs on the float64 pipe.

// Scale exponent s for the fixed-point grid. One atom's weight at a grid point
// is at most 1 and a derivative weight at most sc = K/L in magnitude, so
// |grid value| <= 3 sc m cmax, with m = max |dipole component| and cmax the
// number of atoms that reach one point; s keeps that below 2^61.
__device__ __forceinline__ int fixed_scale_bound(float bound) {  // |grid value| <= bound
  if (!(bound > 0.f) || !(bound < 1e30f)) return 0;  // zero (or non-finite) input
  int e;
  frexpf(bound, &e);  // bound < 2^e
  return max(-60, min(120, 61 - e));
}

__device__ __forceinline__ int fixed_scale(float m, float sc, int cmax) {
  return fixed_scale_bound(3.f * sc * m * (float)cmax);
}

// round(f * 2^s) to the nearest 64-bit integer (ties to even), by the
// conversion instruction: -60 <= s <= 120 makes 2^s an exact float, the
// product is exact while it is a normal float, and fixed_scale keeps it
// below 2^61 in magnitude; products below 2^-126 round to 0 either way.
__device__ __forceinline__ long long to_fixed(float f, int s) {
  return __float2ll_rn(f * __int_as_float((127 + s) << 23));
}

// Q(g) = sum_i mu_i . grad W_i(g) with mu = v32 + vlo. One thread per
// (atom, y row, z point) adds the atom's value at the five x planes, so the
// lanes of a warp that share (atom, y row) hit five consecutive z points:
// the atomics of one row coalesce. vmax[kReduceBlocks] holds max |v32| as left
// by the kernel that split v; every block derives the same scale from it and
// block 0 stores it in fx_info[0] for the FFT.
constexpr int kSpreadThreads = 256;
__global__ void __launch_bounds__(kSpreadThreads) k_spread_dipoles_fx(int n, const float2* __restrict__ th_df,
                                                                      const int4* __restrict__ gbase,
                                                                      const float4* __restrict__ v32,
                                                                      const float4* __restrict__ vlo,
                                                                      const float* __restrict__ vmax,
                                                                      int* __restrict__ fx_info, float sc, int K,
                                                                      unsigned long long* __restrict__ grid,
                                                                      const int* __restrict__ stop) {
  pdl_wait();  // first: a kernel never completes before the one it depends on
  if (stop && *stop) return;
  pdl_trigger();
  const int sfx = fixed_scale(vmax[kReduceBlocks], sc, kOrder * kOrder * kOrder * fx_info[1]);
  if (blockIdx.x == 0 && threadIdx.x == 0) fx_info[0] = sfx;
  const long long item = (long long)blockIdx.x * kSpreadThreads + threadIdx.x;
  if (item >= (long long)n * (kOrder * kOrder)) return;
  const int s = (int)(item / (kOrder * kOrder)), tyz = (int)(item - (long long)s * (kOrder * kOrder));
  const int ty = tyz / kOrder, tz = tyz - ty * kOrder;
  const float2* th = th_df + (long long)kThDf * s;
  const float4 h = v32[s], l = vlo ? vlo[s] : make_float4(0.f, 0.f, 0.f, 0.f);
  const float2 y0 = th[(1 * 2 + 0) * kOrder + ty], y1 = th[(1 * 2 + 1) * kOrder + ty];
  const float2 z0 = th[(2 * 2 + 0) * kOrder + tz], z1 = th[(2 * 2 + 1) * kOrder + tz];
  // P = mu_y w'_y w_z + mu_z w_y w'_z, Q = mu_x w_y w_z: the point's value is P w_x + Q w'_x
  const dflt P = df_madd(df_mul({h.z, l.z}, {y0.x, y0.y}), {z1.x, z1.y},
                         df_mul(df_mul({h.y, l.y}, {y1.x, y1.y}), {z0.x, z0.y}));
  const dflt Q = df_mul(df_mul({h.x, l.x}, {y0.x, y0.y}), {z0.x, z0.y});
  const int4 b = gbase[s];
  unsigned long long* col = grid + (long long)wrapk(b.y - ty, K) * K + wrapk(b.z - tz, K);
  const long long plane = (long long)K * K;
#pragma unroll
  for (int tx = 0; tx < kOrder; ++tx) {
    const float2 x0 = th[(0 * 2 + 0) * kOrder + tx], x1 = th[(0 * 2 + 1) * kOrder + tx];
    const dflt val = df_madd(Q, {x1.x, x1.y}, df_mul(P, {x0.x, x0.y}));
    const long long q = to_fixed(val.hi, sfx) + to_fixed(val.lo, sfx);
    atomicAdd(col + wrapk(b.x - tx, K) * plane, (unsigned long long)q);
  }
}

// fixed-point grid -> float64 grid (for cuFFT), zeroing the fixed-point grid
__global__ void k_fixed_to_double(long long ng, unsigned long long* __restrict__ qfx, const int* __restrict__ fx_info,
                                  double* __restrict__ out, const int* __restrict__ stop) {
  if (stop && *stop) return;
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= ng) return;
  const long long v = (long long)qfx[k];
  qfx[k] = 0ull;
  out[k] = ldexp((double)v, -fx_info[0]);
}

template <typename C, typename R>
__global__ void k_convolve(long long m, C* __restrict__ cg, const R* __restrict__ G,
                           const int* __restrict__ stop = nullptr) {
  if (stop && *stop) return;
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= m) return;
  const R g = G[k];
  C v = cg[k];
  v.x *= g;
  v.y *= g;
  cg[k] = v;
}

// phi = hi + lo for every grid point (float64 path, once per gather)
__global__ void k_split_grid(long long ng, const double* __restrict__ phi, float2* __restrict__ out,
                             const int* __restrict__ stop) {
  if (stop && *stop) return;
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= ng) return;
  const dflt v = df_split(phi[k]);
  out[k] = make_float2(v.hi, v.lo);
}

// The float64 path's gather in double-float arithmetic (float units only):
// weights, their derivatives and the grid potential are hi/lo pairs. Six
// atoms per warp, five lanes each (lanes 30 and 31 idle): lane t of an atom
// sums z plane k0z - t, so the five lanes read five consecutive z points of a
// grid row at a time; they then add their sums in a fixed order.
constexpr int kGatherAtomsPerWarp = 6;
constexpr int kGatherThreads = 128;

__device__ __forceinline__ dflt sum_five(dflt v, int base) {  // same order in all five lanes
  dflt t = {__shfl_sync(0xffffffffu, v.hi, base), __shfl_sync(0xffffffffu, v.lo, base)};
#pragma unroll
  for (int k = 1; k < kOrder; ++k)
    t = df_add(t, {__shfl_sync(0xffffffffu, v.hi, base + k), __shfl_sync(0xffffffffu, v.lo, base + k)});
  return t;
}

template <bool kSet>
__global__ void __launch_bounds__(kGatherThreads) k_gather_field_df(int n, const float2* __restrict__ th_df,
                                                                     const int4* __restrict__ gbase,
                                                                     const float2* __restrict__ phi, int K,
                                                                     double4_32a* __restrict__ out,
                                                                     const int* __restrict__ stop) {
  pdl_wait();  // first: a kernel never completes before the one it depends on
  if (stop && *stop) return;
  pdl_trigger();
  const int lane = threadIdx.x & 31, seg = lane / kOrder, tz = lane - seg * kOrder;
  const int warp = (blockIdx.x * kGatherThreads + threadIdx.x) >> 5;
  const int s = warp * kGatherAtomsPerWarp + seg;
  if (warp * kGatherAtomsPerWarp >= n) return;
  const bool active = seg < kGatherAtomsPerWarp && s < n;
  dflt ex = {0.f, 0.f}, ey = {0.f, 0.f}, ez = {0.f, 0.f};
  if (active) {
    const int4 b = gbase[s];
    const float2* th = th_df + (long long)kThDf * s;
    const float2 wz0 = th[(2 * 2 + 0) * kOrder + tz], wz1 = th[(2 * 2 + 1) * kOrder + tz];
    float2 wx0[kOrder], wx1[kOrder];
    int gx[kOrder];
    for (int t = 0; t < kOrder; ++t) {
      wx0[t] = th[(0 * 2 + 0) * kOrder + t];
      wx1[t] = th[(0 * 2 + 1) * kOrder + t];
      gx[t] = wrapk(b.x - t, K) * K * K;
    }
    const float2* pz = phi + wrapk(b.z - tz, K);
    dflt px = {0.f, 0.f}, py = {0.f, 0.f}, pzz = {0.f, 0.f};
    for (int ty = 0; ty < kOrder; ++ty) {
      const float2 wy0 = th[(1 * 2 + 0) * kOrder + ty], wy1 = th[(1 * 2 + 1) * kOrder + ty];
      const float2* col = pz + wrapk(b.y - ty, K) * K;
      dflt s0 = {0.f, 0.f}, s1 = {0.f, 0.f};
      for (int tx = 0; tx < kOrder; ++tx) {
        const float2 ph = col[gx[tx]];
        df_fma(s0, wx0[tx].x, wx0[tx].y, ph.x, ph.y);
        df_fma(s1, wx1[tx].x, wx1[tx].y, ph.x, ph.y);
      }
      df_fma(px, wy0.x, wy0.y, s1.hi, s1.lo);
      df_fma(py, wy1.x, wy1.y, s0.hi, s0.lo);
      df_fma(pzz, wy0.x, wy0.y, s0.hi, s0.lo);
    }
    ex = df_mul({wz0.x, wz0.y}, px);
    ey = df_mul({wz0.x, wz0.y}, py);
    ez = df_mul({wz1.x, wz1.y}, pzz);
  }
  const int base = min(seg, kGatherAtomsPerWarp - 1) * kOrder;
  ex = sum_five(ex, base);
  ey = sum_five(ey, base);
  ez = sum_five(ez, base);
  if (!active) return;
  double* o = reinterpret_cast<double*>(out + s);
  if (tz < 3) {
    const double f = df_to_double(tz == 0 ? ex : (tz == 1 ? ey : ez));
    if (kSet)
      o[tz] = -f;
    else
      o[tz] -= f;
  } else if (kSet && tz == 3) {
    o[3] = 0.0;
  }
}

// The permanent field's reciprocal part in float64: float64 weights
// (k_theta), float64 grid potential phi (cuFFT), float64 sums. Six atoms per
// warp, five lanes each, as in k_gather_field_df; lane t of an atom sums z
// plane k0z - t, then the five lanes add their sums in a fixed order.
// out = -grad phi at each atom.
__device__ __forceinline__ double sum_five64(double v, int base) {  // same order in all five lanes
  double t = __shfl_sync(0xffffffffu, v, base);
#pragma unroll
  for (int k = 1; k < kOrder; ++k) t += __shfl_sync(0xffffffffu, v, base + k);
  return t;
}

__global__ void __launch_bounds__(kGatherThreads) k_gather_field64(int n, const double* __restrict__ theta,
                                                                    const int4* __restrict__ gbase,
                                                                    const double* __restrict__ phi, int K,
                                                                    double4_32a* __restrict__ out) {
  const int lane = threadIdx.x & 31, seg = lane / kOrder, tz = lane - seg * kOrder;
  const int warp = (blockIdx.x * kGatherThreads + threadIdx.x) >> 5;
  const int s = warp * kGatherAtomsPerWarp + seg;
  if (warp * kGatherAtomsPerWarp >= n) return;
  const bool active = seg < kGatherAtomsPerWarp && s < n;
  double ex = 0.0, ey = 0.0, ez = 0.0;
  if (active) {
    const int4 b = gbase[s];
    const double* th = theta + (long long)kTh * s;
    const double wz0 = th[(2 * 4 + 0) * kOrder + tz], wz1 = th[(2 * 4 + 1) * kOrder + tz];
    double wx0[kOrder], wx1[kOrder];
    int gx[kOrder];
    for (int t = 0; t < kOrder; ++t) {
      wx0[t] = th[(0 * 4 + 0) * kOrder + t];
      wx1[t] = th[(0 * 4 + 1) * kOrder + t];
      gx[t] = wrapk(b.x - t, K) * K * K;
    }
    const double* pz = phi + wrapk(b.z - tz, K);
    double px = 0.0, py = 0.0, pzz = 0.0;
    for (int ty = 0; ty < kOrder; ++ty) {
      const double wy0 = th[(1 * 4 + 0) * kOrder + ty], wy1 = th[(1 * 4 + 1) * kOrder + ty];
      const double* col = pz + wrapk(b.y - ty, K) * K;
      double s0 = 0.0, s1 = 0.0;
      for (int tx = 0; tx < kOrder; ++tx) {
        const double ph = col[gx[tx]];
        s0 = fma(wx0[tx], ph, s0);
        s1 = fma(wx1[tx], ph, s1);
      }
      px = fma(wy0, s1, px);
      py = fma(wy1, s0, py);
      pzz = fma(wy0, s0, pzz);
    }
    ex = wz0 * px;
    ey = wz0 * py;
    ez = wz1 * pzz;
  }
  const int base = min(seg, kGatherAtomsPerWarp - 1) * kOrder;
  ex = sum_five64(ex, base);
  ey = sum_five64(ey, base);
  ez = sum_five64(ez, base);
  if (!active || tz >= 4) return;
  double* o = reinterpret_cast<double*>(out + s);
  o[tz] = tz == 3 ? 0.0 : -(tz == 0 ? ex : (tz == 1 ? ey : ez));
}

// ---- the mixed path's operator: float32 reciprocal chain.
// Spreading of the float32 dipoles v32 with float32 weights (the hi parts of
// theta_df) into the float grid spread32 with float atomics, one thread per
// (atom, y row, z point) over the five x planes, as in k_spread_dipoles_fx.
__global__ void __launch_bounds__(kSpreadThreads) k_spread_dipoles32(int n, const float2* __restrict__ th_df,
                                                                     const int4* __restrict__ gbase,
                                                                     const float4* __restrict__ v32, int K,
                                                                     float* __restrict__ grid,
                                                                     const int* __restrict__ stop) {
  pdl_wait();  // first: a kernel never completes before the one it depends on
  if (stop && *stop) return;
  pdl_trigger();
  const long long item = (long long)blockIdx.x * kSpreadThreads + threadIdx.x;
  if (item >= (long long)n * (kOrder * kOrder)) return;
  const int s = (int)(item / (kOrder * kOrder)), tyz = (int)(item - (long long)s * (kOrder * kOrder));
  const int ty = tyz / kOrder, tz = tyz - ty * kOrder;
  const float2* th = th_df + (long long)kThDf * s;
  const float4 h = v32[s];
  const float y0 = th[(1 * 2 + 0) * kOrder + ty].x, y1 = th[(1 * 2 + 1) * kOrder + ty].x;
  const float z0 = th[(2 * 2 + 0) * kOrder + tz].x, z1 = th[(2 * 2 + 1) * kOrder + tz].x;
  // P = mu_y w'_y w_z + mu_z w_y w'_z, Q = mu_x w_y w_z: the point's value is P w_x + Q w'_x
  const float P = fmaf(h.z * y0, z1, h.y * y1 * z0);
  const float Q = h.x * y0 * z0;
  const int4 b = gbase[s];
  float* col = grid + (long long)wrapk(b.y - ty, K) * K + wrapk(b.z - tz, K);
  const long long plane = (long long)K * K;
#pragma unroll
  for (int tx = 0; tx < kOrder; ++tx) {
    const float x0 = th[(0 * 2 + 0) * kOrder + tx].x, x1 = th[(0 * 2 + 1) * kOrder + tx].x;
    atomicAdd(col + wrapk(b.x - tx, K) * plane, fmaf(Q, x1, P * x0));
  }
}

// Gather of the float32 field from the float potential phi with float32
// weights, six atoms per warp and five lanes each as in k_gather_field_df;
// the field lands in float64 (set: out = -grad phi, else out -= grad phi).
__device__ __forceinline__ float sum_five32(float v, int base) {  // same order in all five lanes
  float t = __shfl_sync(0xffffffffu, v, base);
#pragma unroll
  for (int k = 1; k < kOrder; ++k) t += __shfl_sync(0xffffffffu, v, base + k);
  return t;
}

template <bool kSet>
__global__ void __launch_bounds__(kGatherThreads) k_gather_field32(int n, const float2* __restrict__ th_df,
                                                                    const int4* __restrict__ gbase,
                                                                    const float* __restrict__ phi, int K,
                                                                    double4_32a* __restrict__ out,
                                                                    const int* __restrict__ stop) {
  pdl_wait();  // first: a kernel never completes before the one it depends on
  if (stop && *stop) return;
  pdl_trigger();
  const int lane = threadIdx.x & 31, seg = lane / kOrder, tz = lane - seg * kOrder;
  const int warp = (blockIdx.x * kGatherThreads + threadIdx.x) >> 5;
  const int s = warp * kGatherAtomsPerWarp + seg;
  if (warp * kGatherAtomsPerWarp >= n) return;
  const bool active = seg < kGatherAtomsPerWarp && s < n;
  float ex = 0.f, ey = 0.f, ez = 0.f;
  if (active) {
    const int4 b = gbase[s];
    const float2* th = th_df + (long long)kThDf * s;
    const float wz0 = th[(2 * 2 + 0) * kOrder + tz].x, wz1 = th[(2 * 2 + 1) * kOrder + tz].x;
    float wx0[kOrder], wx1[kOrder];
    int gx[kOrder];
    for (int t = 0; t < kOrder; ++t) {
      wx0[t] = th[(0 * 2 + 0) * kOrder + t].x;
      wx1[t] = th[(0 * 2 + 1) * kOrder + t].x;
      gx[t] = wrapk(b.x - t, K) * K * K;
    }
    const float* pz = phi + wrapk(b.z - tz, K);
    float px = 0.f, py = 0.f, pzz = 0.f;
    for (int ty = 0; ty < kOrder; ++ty) {
      const float wy0 = th[(1 * 2 + 0) * kOrder + ty].x, wy1 = th[(1 * 2 + 1) * kOrder + ty].x;
      const float* col = pz + wrapk(b.y - ty, K) * K;
      float s0 = 0.f, s1 = 0.f;
      for (int tx = 0; tx < kOrder; ++tx) {
        const float ph = col[gx[tx]];
        s0 = fmaf(wx0[tx], ph, s0);
        s1 = fmaf(wx1[tx], ph, s1);
      }
      px = fmaf(wy0, s1, px);
      py = fmaf(wy1, s0, py);
      pzz = fmaf(wy0, s0, pzz);
    }
    ex = wz0 * px;
    ey = wz0 * py;
    ez = wz1 * pzz;
  }
  const int base = min(seg, kGatherAtomsPerWarp - 1) * kOrder;
  ex = sum_five32(ex, base);
  ey = sum_five32(ey, base);
  ez = sum_five32(ez, base);
  if (!active) return;
  double* o = reinterpret_cast<double*>(out + s);
  if (tz < 3) {
    const double f = (double)(tz == 0 ? ex : (tz == 1 ? ey : ez));
    if (kSet)
      o[tz] = -f;
    else
      o[tz] -= f;
  } else if (kSet && tz == 3) {
    o[3] = 0.0;
  }
}

// gather the field in double-float from phi_hi/phi_lo (split = true: first
// split the float64 grid potential in grid64 into them)
template <bool kSet>
void gather_df(amp_ctx* c, cudaStream_t st, double4_32a* out, bool split) {
  const int K = c->K, n = c->n;
  const long long ng = (long long)K * K * K;
  c->n_launch += split ? 2 : 1;
  if (split) k_split_grid<<<amp_blocks(ng, 256), 256, 0, st>>>(ng, c->grid64, c->phi_df, c->op_stop);
  const long long warps = (n + kGatherAtomsPerWarp - 1) / kGatherAtomsPerWarp;
  launch_pdl(k_gather_field_df<kSet>, dim3(amp_blocks(warps * 32, kGatherThreads)), dim3(kGatherThreads), 0, st, n,
             c->theta_df, c->gbase, c->phi_df, K, out, c->op_stop);
}

int exec_fft(amp_ctx* c, bool fp32, bool forward);

// Fixed-point grid gridfx (zeroed on the way) -> phi. The double-float FFT
// writes phi_df directly when the grid size allows it, else cuFFT float64
// leaves phi in grid64 and *split_needed tells the gather to split it first.
int conv_to_phi(amp_ctx* c, cudaStream_t st, bool* split_needed) {
  if (c->fft_grid) {
    fft_df_convolve(c, st);
    *split_needed = false;
    return AMP_OK;
  }
  const long long ng = (long long)c->K * c->K * c->K;
  const long long nh = (long long)c->K * c->K * (c->K / 2 + 1);
  c->n_launch += 2;
  k_fixed_to_double<<<amp_blocks(ng, 256), 256, 0, st>>>(ng, c->gridfx, c->fx_info, c->grid64, c->op_stop);
  cufftSetStream(c->plan_d2z, st);
  cufftSetStream(c->plan_z2d, st);
  int r = exec_fft(c, false, true);
  if (!r) {
    k_convolve<<<amp_blocks(nh, 256), 256, 0, st>>>(nh, c->cgrid64, c->G64, c->op_stop);
    r = exec_fft(c, false, false);
  }
  cufftSetStream(c->plan_d2z, c->stream);
  cufftSetStream(c->plan_z2d, c->stream);
  *split_needed = true;
  return r;
}

// Host: B-spline moduli and influence function, float64.
double m5_at(double u) {  // M5 at integer-shifted u by the recursion (host side)
  // M2 on [0, 2]
  auto M = [](int n, double x, auto&& self) -> double {
    if (n == 2) return x <= 0.0 || x >= 2.0 ? 0.0 : 1.0 - std::fabs(x - 1.0);
    return (x * self(n - 1, x, self) + (n - x) * self(n - 1, x - 1.0, self)) / (n - 1);
  };
  return M(5, u, M);
}

std::vector<double> moduli(int K) {
  std::vector<double> b2(K, 0.0);
  std::vector<char> ok(K, 0);
  for (int m = 0; m < K; ++m) {
    double re = 0, im = 0;
    for (int k = 0; k < kOrder - 1; ++k) {
      const double mk = m5_at(k + 1.0);
      const double ang = 2.0 * M_PI * (double)m * (double)k / (double)K;
      re += mk * std::cos(ang);
      im += mk * std::sin(ang);
    }
    const double den = re * re + im * im;
    if (den >= 1e-7) {
      b2[m] = 1.0 / den;
      ok[m] = 1;
    }
  }
  for (int m = 0; m < K; ++m)
    if (!ok[m]) b2[m] = 0.5 * (b2[(m - 1 + K) % K] + b2[(m + 1) % K]);
  return b2;
}

int exec_fft(amp_ctx* c, bool fp32, bool forward) {
  cufftResult r;
  if (!fp32)
    r = forward ? cufftExecD2Z(c->plan_d2z, c->grid64, reinterpret_cast<cufftDoubleComplex*>(c->cgrid64))
                : cufftExecZ2D(c->plan_z2d, reinterpret_cast<cufftDoubleComplex*>(c->cgrid64), c->grid64);
  else
    r = forward ? cufftExecR2C(c->plan_r2c, c->grid32, reinterpret_cast<cufftComplex*>(c->cgrid32))
                : cufftExecC2R(c->plan_c2r, reinterpret_cast<cufftComplex*>(c->cgrid32), c->grid32);
  if (r != CUFFT_SUCCESS) return fail(c, AMP_ERR_CUDA, "cuFFT exec failed (%d)", (int)r);
  return AMP_OK;
}

// Influence function G(m) on the half spectrum for the current box and
// beta, on the context stream (no host work, no synchronisation):
//   G(m) = exp(-pi^2 m~^2/beta^2) / (pi V m~^2) |b(m1) b(m2) b(m3)|^2, G(0) = 0,
// m~ = (m1, m2, m3)/L with m_a in (-K/2, K/2], index ((mx K + my)(K/2+1) + mz);
// float64, its float copy (mixed path) and its hi/lo split (own FFT).
__global__ void k_influence(int K, double L, double beta, const double* __restrict__ b2, double* __restrict__ G,
                            float* __restrict__ G32, float2* __restrict__ Gdf) {
  const long long nh = (long long)K * K * (K / 2 + 1);
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nh) return;
  const int mz = (int)(k % (K / 2 + 1));
  const long long t = k / (K / 2 + 1);
  const int my = (int)(t % K), mx = (int)(t / K);
  const double fx = (mx <= K / 2 ? mx : mx - K) / L, fy = (my <= K / 2 ? my : my - K) / L, fz = mz / L;
  const double m2 = fx * fx + fy * fy + fz * fz;
  double g = 0.0;
  if (m2 > 0.0)
    g = exp(-M_PI * M_PI * m2 / (beta * beta)) / (M_PI * L * L * L * m2) * b2[mx] * b2[my] * b2[mz];
  G[k] = g;
  if (G32) G32[k] = (float)g;
  if (Gdf) {
    const float h = (float)g;
    Gdf[k] = make_float2(h, (float)(g - (double)h));
  }
}

}  // namespace

int pme_influence(amp_ctx* c) {
  const int K = c->K;
  const long long nh = (long long)K * K * (K / 2 + 1);
  c->n_launch += 1;
  k_influence<<<amp_blocks(nh, 256), 256, 0, c->stream>>>(K, c->cfg.box, c->cfg.ewald_beta, c->bmod, c->G64,
                                                         c->cfg.precision == AMP_MIXED ? c->G32 : nullptr,
                                                         c->fft_grid ? c->fft_G : nullptr);
  return cuda_check(c, cudaGetLastError(), "influence function");
}

int pme_setup(amp_ctx* c) {
  const int K = c->cfg.pme_grid;
  c->K = K;
  const long long ng = (long long)K * K * K, nh = (long long)K * K * (K / 2 + 1);
  int r;
  if ((r = dev_alloc(c, &c->grid64, ng)) || (r = dev_alloc(c, &c->cgrid64, nh)) ||
      (r = dev_alloc(c, &c->G64, nh)))
    return r;
  // the reciprocal part of both precisions: fixed-point grid, double-float
  // transform and gather (the mixed path's float32 grids serve its forces)
  if ((r = dev_alloc(c, &c->phi_df, ng)) || (r = dev_alloc(c, &c->gridfx, ng)) ||
      (r = dev_alloc(c, &c->kcount, ng)) || (r = dev_alloc(c, &c->fx_info, 4)))
    return r;
  // the fixed-point grid starts at zero; the kernel that reads it zeroes it again
  if ((r = cuda_check(c, cudaMemsetAsync(c->gridfx, 0, sizeof(unsigned long long) * ng, c->stream),
                      "grid memset")))
    return r;
  if (c->cfg.precision == AMP_MIXED) {
    if ((r = dev_alloc(c, &c->grid32, ng)) || (r = dev_alloc(c, &c->cgrid32, nh)) ||
        (r = dev_alloc(c, &c->G32, nh)) || (r = dev_alloc(c, &c->spread32, ng)) || (r = dev_alloc(c, &c->phi32, ng)))
      return r;
    // the operator's float32 spreading grid starts at zero; the own FFT's
    // first pass zeroes what it reads, the cuFFT path clears it before use
    if ((r = cuda_check(c, cudaMemsetAsync(c->spread32, 0, sizeof(float) * ng, c->stream), "grid memset")))
      return r;
  }
  if (fft_own_supported(K)) {
    // the permanent field's float64 grids for the own FFT; its first pass
    // zeroes the spreading grid as it reads it, so it stays zero between uses
    if ((r = dev_alloc(c, &c->spread64, ng)) || (r = dev_alloc(c, &c->phi64, ng))) return r;
    if ((r = cuda_check(c, cudaMemsetAsync(c->spread64, 0, sizeof(double) * ng, c->stream), "grid memset")))
      return r;
  }
  {  // B-spline moduli |b(m)|^2 (they depend on K only)
    const std::vector<double> b2 = moduli(K);
    if ((r = dev_alloc(c, &c->bmod, K)) ||
        (r = cuda_check(c, cudaMemcpyAsync(c->bmod, b2.data(), sizeof(double) * K, cudaMemcpyHostToDevice, c->stream),
                        "moduli upload")))
      return r;
  }
  if (fft_own_supported(K) && (r = fft_own_setup(c))) return r;
  if ((r = pme_influence(c))) return r;
  if (cufftPlan3d(&c->plan_d2z, K, K, K, CUFFT_D2Z) != CUFFT_SUCCESS ||
      cufftPlan3d(&c->plan_z2d, K, K, K, CUFFT_Z2D) != CUFFT_SUCCESS)
    return fail(c, AMP_ERR_CUDA, "cuFFT plan creation failed");
  cufftSetStream(c->plan_d2z, c->stream);
  cufftSetStream(c->plan_z2d, c->stream);
  if (c->cfg.precision == AMP_MIXED) {
    if (cufftPlan3d(&c->plan_r2c, K, K, K, CUFFT_R2C) != CUFFT_SUCCESS ||
        cufftPlan3d(&c->plan_c2r, K, K, K, CUFFT_C2R) != CUFFT_SUCCESS)
      return fail(c, AMP_ERR_CUDA, "cuFFT plan creation failed");
    cufftSetStream(c->plan_r2c, c->stream);
    cufftSetStream(c->plan_c2r, c->stream);
  }
  c->plans = true;
  return AMP_OK;
}

int pme_alloc_atoms(amp_ctx* c, int n_cap) {
  int r;
  if ((r = dev_alloc(c, &c->theta, (long long)kTh * n_cap)) || (r = dev_alloc(c, &c->gbase, n_cap))) return r;
  if (c->cfg.precision == AMP_MIXED && (r = dev_alloc(c, &c->theta32, (long long)kTh * n_cap))) return r;
  if ((r = dev_alloc(c, &c->theta_df, (long long)kThDf * n_cap))) return r;
  return AMP_OK;
}

// B-spline weights of the current system in double-float (k_theta_df), for
// the dipole products of both precisions, on stream st. The float64 copy
// (and the mixed path's float32 one), which the permanent field and the
// force kernels read, come from pme_theta64.
void launch_pme_theta(amp_ctx* c, cudaStream_t st) {
  c->n_launch += 1;
  cudaMemsetAsync(c->kcount, 0, sizeof(int) * (long long)c->K * c->K * c->K, st);
  cudaMemsetAsync(c->fx_info, 0, sizeof(int) * 4, st);
  const double sc = (double)c->K / c->cfg.box;
  const float sh = (float)sc;
  k_theta_df<<<amp_blocks(4LL * c->n, 128), 128, 0, st>>>(c->n, c->atomA, c->cfg.box, c->K,
                                                         make_float2(sh, (float)(sc - (double)sh)), c->theta_df,
                                                         c->gbase, c->kcount, c->fx_info);
  c->theta64_valid = false;
}

void pme_theta64(amp_ctx* c, cudaStream_t st) {
  if (c->theta64_valid) return;
  c->n_launch += 1;
  k_theta<<<amp_blocks(3LL * c->n, 128), 128, 0, st>>>(c->n, c->atomA, c->cfg.box, c->K, c->theta, c->theta32);
  c->theta64_valid = true;
}

// The geometry-dependent reciprocal-space work of a new system, on the side
// stream so that it runs beside the neighbour search, the pair build and the
// real-space permanent field of the main stream (it keeps the float64 pipe
// busy, they the float32 one): the B-spline weights (double-float, float64), then the permanent
// field's reciprocal part into e0rec. That part is float64 throughout: in a
// system whose molecules are far apart the excluded intramolecular
// real-space terms and this part (each ~1e-1 e/A^2) cancel to a field ~1e-4,
// so both are computed in float64 and meet in float64 (k_intra_fields64 for
// the excluded terms). Float64 multipole spreading (atomics), cuFFT float64,
// float64 gather. Every later call waits for it (join_geometry).
int pme_geometry(amp_ctx* c) {
  cudaEventRecord(c->ev_fork, c->stream);
  cudaStreamWaitEvent(c->side, c->ev_fork, 0);
  int r = AMP_OK;
  {
    PhaseScope ps(c, AMP_PHASE_E0_RECIP, c->side);
    launch_pme_theta(c, c->side);
    pme_theta64(c, c->side);
    const double* phi = c->grid64;
    if (c->fft_grid64) {  // a grid of the own FFT: its float64 variant, which zeroes spread64 as it reads it
      c->n_launch += 1;
      k_spread_multipoles64<<<amp_blocks((long long)c->n * kOrder * kOrder, 256), 256, 0, c->side>>>(
          c->n, c->theta, c->gbase, c->atomA, c->atomB, c->atomC, c->atomD, c->K, c->spread64);
      fft_f64_convolve(c, c->side, c->spread64, c->phi64);
      phi = c->phi64;
    } else {
      r = pme_potential(c, false, true, nullptr, nullptr, c->grid64, c->side);
    }
    if (!r) {
      const long long warps = (c->n + kGatherAtomsPerWarp - 1) / kGatherAtomsPerWarp;
      c->n_launch += 1;
      k_gather_field64<<<amp_blocks(warps * 32, kGatherThreads), kGatherThreads, 0, c->side>>>(
          c->n, c->theta, c->gbase, phi, c->K, c->e0rec);
    }
  }
  cudaEventRecord(c->ev_geom, c->side);
  c->geom_pending = true;
  return r;
}

// Grid potential phi = conv(Q) into grid_out (float64 or float32 grid), Q the
// spread of the dipoles v (v32 in float32) or of the permanent multipoles.
int pme_potential(amp_ctx* c, bool fp32, bool multipoles, const double4_32a* v, const float4* v32, void* grid_out,
                  cudaStream_t st) {
  const int K = c->K, n = c->n;
  const long long ng = (long long)K * K * K, nh = (long long)K * K * (K / 2 + 1);
  const int blocks = amp_blocks((long long)n * kPmeGroup, 128);
  c->n_launch += 2;
  cufftResult fr;
  cufftSetStream(fp32 ? c->plan_r2c : c->plan_d2z, st);
  cufftSetStream(fp32 ? c->plan_c2r : c->plan_z2d, st);
  if (!fp32) {
    double* g = static_cast<double*>(grid_out);
    cudaMemsetAsync(g, 0, sizeof(double) * ng, st);
    if (multipoles)
      k_spread_multipoles64<<<amp_blocks((long long)n * kOrder * kOrder, 256), 256, 0, st>>>(
          n, c->theta, c->gbase, c->atomA, c->atomB, c->atomC, c->atomD, K, g);
    else
      k_spread_dipoles<double, double4_32a><<<blocks, 128, 0, st>>>(n, c->theta, c->gbase, v, K, g);
    fr = cufftExecD2Z(c->plan_d2z, g, reinterpret_cast<cufftDoubleComplex*>(c->cgrid64));
    if (fr == CUFFT_SUCCESS) {
      k_convolve<<<amp_blocks(nh, 256), 256, 0, st>>>(nh, c->cgrid64, c->G64);
      fr = cufftExecZ2D(c->plan_z2d, reinterpret_cast<cufftDoubleComplex*>(c->cgrid64), g);
    }
  } else {
    float* g = static_cast<float*>(grid_out);
    cudaMemsetAsync(g, 0, sizeof(float) * ng, st);
    if (multipoles)
      k_spread_multipoles<float><<<blocks, 128, 0, st>>>(n, c->theta32, c->gbase, c->atomA, c->atomB, c->atomC,
                                                         c->atomD, K, g);
    else
      k_spread_dipoles<float, float4><<<blocks, 128, 0, st>>>(n, c->theta32, c->gbase, v32, K, g);
    fr = cufftExecR2C(c->plan_r2c, g, reinterpret_cast<cufftComplex*>(c->cgrid32));
    if (fr == CUFFT_SUCCESS) {
      k_convolve<<<amp_blocks(nh, 256), 256, 0, st>>>(nh, c->cgrid32, c->G32);
      fr = cufftExecC2R(c->plan_c2r, reinterpret_cast<cufftComplex*>(c->cgrid32), g);
    }
  }
  cufftSetStream(fp32 ? c->plan_r2c : c->plan_d2z, c->stream);
  cufftSetStream(fp32 ? c->plan_c2r : c->plan_z2d, c->stream);
  if (fr != CUFFT_SUCCESS) return fail(c, AMP_ERR_CUDA, "cuFFT exec failed (%d)", (int)fr);
  return AMP_OK;
}

// Reciprocal field of the dipoles v on stream st: out (+)= -grad phi. With
// set = true the result overwrites out (used when it runs beside the real-space
// kernel on a second stream and is summed later). The dipoles come as their
// float split, v32 + vlo (vlo null: v32 alone, the mixed path's operator
// input), with the per-block maxima that the splitting kernel left in
// vmax_part.
int pme_dipole_field(amp_ctx* c, const double4_32a* v, const float4* v32, const float4* vlo, double4_32a* out,
                     cudaStream_t st, bool set) {
  (void)v;
  const int K = c->K, n = c->n;
  c->n_launch += 3;  // spread, convolve, gather (cuFFT kernels not counted)
  if (!v32) return fail(c, AMP_ERR_STATE, "reciprocal field needs the float split of the vector");
  {
    PhaseScope ps(c, AMP_PHASE_T_SPREAD, st);
    // an ordinary launch: the chain starts behind an event wait (the fork),
    // and nothing should depend on how a dependent launch treats one
    k_spread_dipoles_fx<<<amp_blocks((long long)n * kOrder * kOrder, kSpreadThreads), kSpreadThreads, 0, st>>>(
        n, c->theta_df, c->gbase, v32, vlo, c->vmax_part, c->fx_info, (float)((double)K / c->cfg.box), K,
        c->gridfx, c->op_stop);
  }
  if (c->spread_event) cudaEventRecord(c->ev_spread, st);
  bool split = true;
  int r;
  {
    PhaseScope ps(c, AMP_PHASE_T_FFT, st);
    r = conv_to_phi(c, st, &split);
  }
  if (r) return r;
  PhaseScope ps(c, AMP_PHASE_T_GATHER, st);
  if (set)
    gather_df<true>(c, st, out, split);
  else
    gather_df<false>(c, st, out, split);
  return AMP_OK;
}

// Reciprocal field of the float32 dipoles v32 in float32 (the mixed path's
// operator; its float64 residual check takes the double-float chain): float
// atomics into spread32, the own float32 FFT on its grids up to kOwnF32MaxK
// (which zeroes spread32 as it reads it), else cuFFT R2C / C2R float32 with
// spread32 cleared first, then the float32 gather; out (+)= -grad phi.
int pme_dipole_field32(amp_ctx* c, const float4* v32, double4_32a* out, cudaStream_t st, bool set) {
  const int K = c->K, n = c->n;
  const long long ng = (long long)K * K * K, nh = (long long)K * K * (K / 2 + 1);
  const bool own = c->fft_grid32 != nullptr;
  int r = AMP_OK;
  if (!own) cudaMemsetAsync(c->spread32, 0, sizeof(float) * ng, st);
  c->n_launch += 2;
  {
    PhaseScope ps(c, AMP_PHASE_T_SPREAD, st);
    k_spread_dipoles32<<<amp_blocks((long long)n * kOrder * kOrder, kSpreadThreads), kSpreadThreads, 0, st>>>(
        n, c->theta_df, c->gbase, v32, K, c->spread32, c->op_stop);
  }
  if (c->spread_event) cudaEventRecord(c->ev_spread, st);
  {
    PhaseScope pf(c, AMP_PHASE_T_FFT, st);
    if (own) {
      fft_f32_convolve(c, st);
    } else {
      c->n_launch += 1;
      cufftSetStream(c->plan_r2c, st);
      cufftSetStream(c->plan_c2r, st);
      cufftResult fr = cufftExecR2C(c->plan_r2c, c->spread32, reinterpret_cast<cufftComplex*>(c->cgrid32));
      if (fr == CUFFT_SUCCESS) {
        k_convolve<<<amp_blocks(nh, 256), 256, 0, st>>>(nh, c->cgrid32, c->G32, c->op_stop);
        fr = cufftExecC2R(c->plan_c2r, reinterpret_cast<cufftComplex*>(c->cgrid32), c->phi32);
      }
      cufftSetStream(c->plan_r2c, c->stream);
      cufftSetStream(c->plan_c2r, c->stream);
      if (fr != CUFFT_SUCCESS) r = fail(c, AMP_ERR_CUDA, "cuFFT exec failed (%d)", (int)fr);
    }
  }
  if (r) return r;
  const long long warps = (n + kGatherAtomsPerWarp - 1) / kGatherAtomsPerWarp;
  const dim3 grid(amp_blocks(warps * 32, kGatherThreads));
  PhaseScope pg(c, AMP_PHASE_T_GATHER, st);
  if (set)
    launch_pdl(k_gather_field32<true>, grid, dim3(kGatherThreads), 0, st, n, c->theta_df, c->gbase, c->phi32, K, out,
               c->op_stop);
  else
    launch_pdl(k_gather_field32<false>, grid, dim3(kGatherThreads), 0, st, n, c->theta_df, c->gbase, c->phi32, K,
               out, c->op_stop);
  return AMP_OK;
}

}  // namespace amp
