// Permanent-multipole energy and its gradients: the interaction of the
// permanent multipoles with each other, the paper's "empole1" (Section
// "Hotspots": the second electrostatic routine of an AMOEBA step beside the
// polarization ones). Charges, dipoles and traceless quadrupoles in the global
// frame, so there are no torques. The pair terms run in double-float on the
// float32 units (no float64 instruction: GB300's float64 rate is 1/64 of its
// float32 rate), the reciprocal gather and the per-atom epilogue in float64.
//
// Real space, unique pair (i, j), r = x_i - x_j (minimum image), kernels
// b_n = B_n (Ewald-screened) or B_n - bare_n for two sites of one molecule
// (the pair is excluded), no Thole damping. With dir = d_i.r, djr = d_j.r,
// ti = Theta_i r, tj = Theta_j r, tir = r.ti, tjr = r.tj, expanding
// (q_i + d_i.grad + Theta_i:grad grad/3)(q_j - d_j.grad + Theta_j:grad grad/3) B_0
// with grad B_n = -r B_{n+1} gives U_ij = sum_n b_n G_n,
//   G0 = q_i q_j
//   G1 = q_i djr - q_j dir + d_i.d_j
//   G2 = -dir djr + (q_i tjr + q_j tir)/3 + 2/3 (d_i.tj - d_j.ti) + 2/9 Theta_i:Theta_j
//   G3 = (djr tir - dir tjr)/3 - 4/9 ti.tj
//   G4 = tir tjr/9,
// and the force on i, -dU_ij/dr = r sum_n G_n b_{n+1} - sum_n b_n grad G_n.
// The derivatives of U_ij in the moments of i are the potential of j at i,
// its gradient and (per quadrupole number) the matching G-terms; those of j
// follow from the same expressions with i and j swapped and r -> -r.
// Reciprocal space: phi = conv(spread(q, d, Theta)) on the float64 grid; per
// atom the interpolated derivatives of orders 0..3 give dU/dq = phi,
// dU/dd = grad phi, dU/dTheta_ab = (grad grad phi)_ab/3 and the force
// -(q grad phi + d.grad grad phi + Theta:grad grad grad phi/3).
// Self: dU/dq = -2 beta/sqrt(pi) q, dU/dd = -(2 beta/sqrt(pi))(2 beta^2/3) d,
// dU/dTheta_ab = -(2 beta/sqrt(pi))(8 beta^4/45) Theta_ab; neutralising
// background: dU/dq = -pi Q_tot/(V beta^2). All in units of C.
// Quadrupole gradients are per stored number (off-diagonals doubled) with the
// mean of the diagonal removed (only traceless changes exist). The energy is
// U = 1/2 sum_i (q_i dU/dq_i + d_i.dU/dd_i + Theta_i.dU/dTheta_i), exact
// because U is a quadratic form in the moments; the per-atom terms are summed
// in a fixed order.
#include "amp_internal.cuh"

namespace amp {
namespace {

constexpr int kGroup = 8;  // lanes per atom in the reciprocal gather (one per x plane)
constexpr int kTh = 3 * 4 * kOrder;

// ---- double-float arithmetic with operators (the pair kernel issues no
// float64 instruction: inputs come pre-split, outputs stay split)
struct D2 {
  dflt v;
};
__device__ __forceinline__ D2 operator+(D2 a, D2 b) { return {df_add(a.v, b.v)}; }
__device__ __forceinline__ D2 operator-(D2 a, D2 b) { return {df_sub(a.v, b.v)}; }
__device__ __forceinline__ D2 operator*(D2 a, D2 b) { return {df_mul(a.v, b.v)}; }
__device__ __forceinline__ D2 operator-(D2 a) { return {df_neg(a.v)}; }
__device__ __forceinline__ D2 num(float x) { return {{x, 0.f}}; }  // exactly representable
__device__ __forceinline__ D2 twice(D2 a) { return {{2.f * a.v.hi, 2.f * a.v.lo}}; }

// 1/3, 2/3, 1/9, 2/9, 4/9 as hi + lo (rounded at compile time)
constexpr float kC3h = (float)(1.0 / 3.0), kC3l = (float)(1.0 / 3.0 - (double)(float)(1.0 / 3.0));
constexpr float kC23h = (float)(2.0 / 3.0), kC23l = (float)(2.0 / 3.0 - (double)(float)(2.0 / 3.0));
constexpr float kC9h = (float)(1.0 / 9.0), kC9l = (float)(1.0 / 9.0 - (double)(float)(1.0 / 9.0));
constexpr float kC29h = (float)(2.0 / 9.0), kC29l = (float)(2.0 / 9.0 - (double)(float)(2.0 / 9.0));
constexpr float kC49h = (float)(4.0 / 9.0), kC49l = (float)(4.0 / 9.0 - (double)(float)(4.0 / 9.0));

struct MGeomDf {
  dflt L, beta, twob2, gpre;
  float invL;
};

// minimum-image component: the pair lies within rc < L/2, so rounding d/L
// from the hi part picks the same image as exact arithmetic would
__device__ __forceinline__ D2 min_image(D2 d, const MGeomDf& g) {
  const float sh = rintf(d.v.hi * g.invL);
  return sh == 0.f ? d : d - num(sh) * D2{g.L};
}

// Theta (xx, yy, zz, xy, xz, yz) times v
__device__ __forceinline__ void th_mul(const D2* t, const D2* v, D2* o) {
  o[0] = t[0] * v[0] + t[3] * v[1] + t[4] * v[2];
  o[1] = t[3] * v[0] + t[1] * v[1] + t[5] * v[2];
  o[2] = t[4] * v[0] + t[5] * v[1] + t[2] * v[2];
}

__device__ __forceinline__ D2 dot3(const D2* a, const D2* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

// row a of Theta times v
__device__ __forceinline__ D2 th_row(const D2* t, int a, const D2* v) {
  const int k0 = a == 0 ? 0 : (a == 1 ? 3 : 4), k1 = a == 0 ? 3 : (a == 1 ? 1 : 5), k2 = a == 0 ? 4 : (a == 1 ? 5 : 2);
  return t[k0] * v[0] + t[k1] * v[1] + t[k2] * v[2];
}

__device__ __forceinline__ void put(float2* o, D2 v) { *o = make_float2(v.v.hi, v.v.lo); }

// Derivatives of the pair energy in the moments of the field-point site, for
// a source (q, d, Theta) at displacement r (field point minus source):
//   o[0]    = q b0 + (d.r) b1 + (r.Th.r) b2/3
//   o[1..3] = -q b1 r + b1 d - (d.r) b2 r + 2/3 b2 Th r - (r.Th.r) b3 r/3
//   o[4..9] = E_ab for ab = xx, yy, zz, xy, xz, yz (off-diagonals doubled),
//     E_ab = b2 [q r_a r_b/3 - (d_a r_b + d_b r_a)/3 + 2/9 Th_ab]
//          + b3 [(d.r) r_a r_b/3 - 2/9 (r_a (Th r)_b + (Th r)_a r_b)] + b4 (r.Th.r) r_a r_b/9
__device__ __forceinline__ void moment_jet(const D2* r, D2 q, const D2* d, const D2* th, const D2* b, D2* o) {
  const D2 third = {{kC3h, kC3l}}, two3 = {{kC23h, kC23l}}, ninth = {{kC9h, kC9l}}, two9 = {{kC29h, kC29l}};
  D2 t[3];
  th_mul(th, r, t);
  const D2 dr = dot3(d, r), trr = dot3(t, r);
  o[0] = q * b[0] + dr * b[1] + trr * b[2] * third;
  const D2 rad = -(q * b[1] + dr * b[2] + trr * b[3] * third);
  const D2 b2t = b[2] * two3;
#pragma unroll
  for (int a = 0; a < 3; ++a) o[1 + a] = rad * r[a] + b[1] * d[a] + b2t * t[a];
  const int ia[6] = {0, 1, 2, 0, 0, 1}, ib[6] = {0, 1, 2, 1, 2, 2};
  const D2 c0 = (b[2] * q + b[3] * dr) * third + b[4] * trr * ninth;
  const D2 c1 = b[2] * third, c2 = b[2] * two9, c3 = b[3] * two9;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const int a = ia[k], bb = ib[k];
    const D2 e = c0 * r[a] * r[bb] - c1 * (d[a] * r[bb] + d[bb] * r[a]) + c2 * th[k] -
                 c3 * (r[a] * t[bb] + t[a] * r[bb]);
    o[4 + k] = k < 3 ? e : twice(e);
  }
}

// -dU_ij/dr (the force on i) = r sum_n G_n b_{n+1} - sum_n b_n grad G_n
__device__ __forceinline__ void pair_force(const D2* r, const D2* b, D2 qi, const D2* dpi, const D2* thi, D2 qj,
                                           const D2* dpj, const D2* thj, D2* f) {
  const D2 third = {{kC3h, kC3l}}, two3 = {{kC23h, kC23l}}, ninth = {{kC9h, kC9l}}, two9 = {{kC29h, kC29l}},
           four9 = {{kC49h, kC49l}};
  D2 ti[3], tj[3];
  th_mul(thi, r, ti);
  th_mul(thj, r, tj);
  const D2 dir = dot3(dpi, r), djr = dot3(dpj, r), tir = dot3(ti, r), tjr = dot3(tj, r);
  const D2 thth = thi[0] * thj[0] + thi[1] * thj[1] + thi[2] * thj[2] +
                  twice(thi[3] * thj[3] + thi[4] * thj[4] + thi[5] * thj[5]);
  const D2 G0 = qi * qj;
  const D2 G1 = qi * djr - qj * dir + dot3(dpi, dpj);
  const D2 G2 = (qi * tjr + qj * tir) * third - dir * djr + (dot3(dpi, tj) - dot3(dpj, ti)) * two3 + thth * two9;
  const D2 G3 = (djr * tir - dir * tjr) * third - dot3(ti, tj) * four9;
  const D2 G4 = tir * tjr * ninth;
  const D2 rad = G0 * b[1] + G1 * b[2] + G2 * b[3] + G3 * b[4] + G4 * b[5];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const D2 g1 = qi * dpj[a] - qj * dpi[a];
    const D2 g2 = (qi * tj[a] + qj * ti[a] + th_row(thj, a, dpi) - th_row(thi, a, dpj)) * two3 -
                  (dpi[a] * djr + dpj[a] * dir);
    const D2 g3 = (dpj[a] * tir + twice(djr * ti[a]) - twice(tj[a] * dir) - tjr * dpi[a]) * third -
                  (th_row(thi, a, tj) + th_row(thj, a, ti)) * four9;
    const D2 g4 = (ti[a] * tjr + tj[a] * tir) * two9;
    f[a] = rad * r[a] - (b[1] * g1 + b[2] * g2 + b[3] * g3 + b[4] * g4);
  }
}

// Split moments of atom s: (q, dx), (dy, dz), (Qxx, Qyy), (Qzz, Qxy), (Qxz, Qyz) as hi/lo
struct Moments {
  D2 q, d[3], th[6];
};

__device__ __forceinline__ Moments load_moments(const float4* __restrict__ mp, int s) {
  const float4* m = mp + 5 * (long long)s;
  const float4 m0 = m[0], m1 = m[1], m2 = m[2], m3 = m[3], m4 = m[4];
  Moments o;
  o.q = {{m0.x, m0.y}};
  o.d[0] = {{m0.z, m0.w}};
  o.d[1] = {{m1.x, m1.y}};
  o.d[2] = {{m1.z, m1.w}};
  o.th[0] = {{m2.x, m2.y}};
  o.th[1] = {{m2.z, m2.w}};
  o.th[2] = {{m3.x, m3.y}};
  o.th[3] = {{m3.z, m3.w}};
  o.th[4] = {{m4.x, m4.y}};
  o.th[5] = {{m4.z, m4.w}};
  return o;
}

// One thread per unique pair, in double-float: the force on i (F_j = -F_i)
// and the moment derivatives of both ends, as the per-pair record of 24
// (hi, lo) pairs [force(3), unused, i's derivatives(10), j's derivatives(10)],
// units of C. Inputs: pd = split positions (and molecule), mp = split
// moments, tab = the double-float function table.
__global__ void __launch_bounds__(128) k_mpole_pairs_df(long long nh, const int* __restrict__ half_i,
                                                        const int* __restrict__ half_j,
                                                        const float4* __restrict__ pd,
                                                        const float4* __restrict__ mp, MGeomDf g,
                                                        const float2* __restrict__ tab, float2* __restrict__ out) {
  const long long pid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (pid >= nh) return;
  const int i = half_i[pid], j = half_j[pid];
  const float4 hi_i = pd[3 * (long long)i], lo_i = pd[3 * (long long)i + 1], th_i = pd[3 * (long long)i + 2];
  const float4 hi_j = pd[3 * (long long)j], lo_j = pd[3 * (long long)j + 1], th_j = pd[3 * (long long)j + 2];
  const D2 r[3] = {min_image(D2{{hi_i.x, lo_i.x}} - D2{{hi_j.x, lo_j.x}}, g),
                   min_image(D2{{hi_i.y, lo_i.y}} - D2{{hi_j.y, lo_j.y}}, g),
                   min_image(D2{{hi_i.z, lo_i.z}} - D2{{hi_j.z, lo_j.z}}, g)};
  const D2 nr[3] = {-r[0], -r[1], -r[2]};
  const D2 r2 = dot3(r, r);
  const D2 ir = {df_rsqrt(r2.v)};
  const D2 br = D2{g.beta} * (r2 * ir);
  const D2 e2 = {df_exp_neg((br * br).v, tab)};  // exp(-beta^2 r^2)
  const D2 ir2 = ir * ir;
  D2 b[6];
  b[0] = D2{df_erfcx(br.v, tab)} * e2 * ir;  // erfc(beta r)/r
  D2 fac = e2 * D2{g.gpre};
#pragma unroll
  for (int n = 1; n < 6; ++n) {
    b[n] = (num((float)(2 * n - 1)) * b[n - 1] + fac) * ir2;
    fac = fac * D2{g.twob2};
  }
  if (__float_as_int(th_i.z) == __float_as_int(th_j.z)) {  // same molecule: remove the bare kernels
    D2 e = ir;
    b[0] = b[0] - e;
#pragma unroll
    for (int n = 1; n < 6; ++n) {
      e = e * num((float)(2 * n - 1)) * ir2;
      b[n] = b[n] - e;
    }
  }
  const Moments mi = load_moments(mp, i), mj = load_moments(mp, j);
  float2* o = out + (long long)kForcePairStride * pid;
  D2 v[10];
  pair_force(r, b, mi.q, mi.d, mi.th, mj.q, mj.d, mj.th, v);
#pragma unroll
  for (int a = 0; a < 3; ++a) put(o + a, v[a]);
  o[3] = make_float2(0.f, 0.f);
  moment_jet(r, mj.q, mj.d, mj.th, b, v);  // at i, of j
#pragma unroll
  for (int k = 0; k < 10; ++k) put(o + 4 + k, v[k]);
  moment_jet(nr, mi.q, mi.d, mi.th, b, v);  // at j, of i
#pragma unroll
  for (int k = 0; k < 10; ++k) put(o + 14 + k, v[k]);
}

// Float64 epilogue of one atom's 13 sums (force, q, d, Theta): times C, the
// quadrupole diagonal projected onto traceless changes, outputs in caller
// order, per-atom energy 1/2 (q dU/dq + d.dU/dd + Theta.dU/dTheta).
__device__ __forceinline__ void finish_atom(double* v, const double4_32a& a, const double4_32a& b,
                                            const double4_32a& c, const double4_32a& d, int o, double* F, double* gq,
                                            double* gd, double* gt, double* e_atom, int i) {
  const double th[6] = {c.x, c.y, c.z, c.w, d.x, d.y};
  const double mean = (v[7] + v[8] + v[9]) * (1.0 / 3.0);
  v[7] -= mean;
  v[8] -= mean;
  v[9] -= mean;
  double u = a.w * v[3] + b.x * v[4] + b.y * v[5] + b.z * v[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) u += th[k] * v[7 + k];
  e_atom[i] = 0.5 * u;
  if (F)
    for (int k = 0; k < 3; ++k) F[3 * o + k] = v[k];
  if (gq) gq[o] = v[3];
  if (gd)
    for (int k = 0; k < 3; ++k) gd[3 * o + k] = v[4 + k];
  if (gt)
    for (int k = 0; k < 6; ++k) gt[6 * o + k] = v[7 + k];
}

// Isolated clusters (no box): every pair with the bare kernels b_n = bare_n;
// pairs inside one molecule are skipped (B_n - bare_n vanishes at beta = 0).
// One thread per atom i visits every j (warp-uniform loads) and sums the force
// on i and i's moment derivatives in double-float; no reciprocal, self or
// background terms.
__global__ void __launch_bounds__(128) k_mpole_cluster_df(int n, const float4* __restrict__ pd,
                                                          const float4* __restrict__ mp,
                                                          const double4_32a* __restrict__ A,
                                                          const double4_32a* __restrict__ B,
                                                          const double4_32a* __restrict__ C,
                                                          const double4_32a* __restrict__ D,
                                                          const int* __restrict__ perm, double* __restrict__ F,
                                                          double* __restrict__ gq, double* __restrict__ gd,
                                                          double* __restrict__ gt, double* __restrict__ e_atom) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 hi_i = pd[3 * (long long)i], lo_i = pd[3 * (long long)i + 1], th_i = pd[3 * (long long)i + 2];
  const Moments mi = load_moments(mp, i);
  D2 acc[13];
#pragma unroll
  for (int k = 0; k < 13; ++k) acc[k] = num(0.f);
  for (int j = 0; j < n; ++j) {
    const float4 th_j = pd[3 * (long long)j + 2];
    if (__float_as_int(th_i.z) == __float_as_int(th_j.z)) continue;  // same molecule (and j == i)
    const float4 hi_j = pd[3 * (long long)j], lo_j = pd[3 * (long long)j + 1];
    const D2 r[3] = {D2{{hi_i.x, lo_i.x}} - D2{{hi_j.x, lo_j.x}}, D2{{hi_i.y, lo_i.y}} - D2{{hi_j.y, lo_j.y}},
                     D2{{hi_i.z, lo_i.z}} - D2{{hi_j.z, lo_j.z}}};
    const D2 ir = {df_rsqrt(dot3(r, r).v)};
    const D2 ir2 = ir * ir;
    D2 b[6];
    b[0] = ir;
#pragma unroll
    for (int k = 1; k < 6; ++k) b[k] = b[k - 1] * num((float)(2 * k - 1)) * ir2;
    const Moments mj = load_moments(mp, j);
    D2 v[10];
    pair_force(r, b, mi.q, mi.d, mi.th, mj.q, mj.d, mj.th, v);
#pragma unroll
    for (int a = 0; a < 3; ++a) acc[a] = acc[a] + v[a];
    moment_jet(r, mj.q, mj.d, mj.th, b, v);
#pragma unroll
    for (int k = 0; k < 10; ++k) acc[3 + k] = acc[3 + k] + v[k];
  }
  double v[13];
#pragma unroll
  for (int k = 0; k < 13; ++k) v[k] = df_to_double(acc[k].v) * kCoulomb;
  finish_atom(v, A[i], B[i], C[i], D[i], perm[i], F, gq, gd, gt, e_atom, i);
}

__device__ __forceinline__ unsigned group_mask() {
  return ((1u << kGroup) - 1u) << ((threadIdx.x & 31) & ~(kGroup - 1));
}

// Reciprocal part per atom: interpolated derivatives of orders 0..3 of the
// permanent-multipole grid potential, then the force and the moment
// derivatives into the per-atom record [force(3), q, d(3), Theta(6)], units of C.
__global__ void __launch_bounds__(128) k_recip_mpole(int n, const double* __restrict__ theta,
                                                     const int4* __restrict__ gbase, const double* __restrict__ phi,
                                                     int K, const double4_32a* __restrict__ A,
                                                     const double4_32a* __restrict__ B,
                                                     const double4_32a* __restrict__ C,
                                                     const double4_32a* __restrict__ D, double* __restrict__ out) {
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  const int s = gid / kGroup, tx = gid % kGroup;
  if (s >= n) return;
  double v[4][4][4];
  #pragma unroll
  for (int a = 0; a < 4; ++a)
    #pragma unroll
    for (int b = 0; b < 4; ++b)
      #pragma unroll
      for (int c = 0; c < 4; ++c) v[a][b][c] = 0.0;
  if (tx < kOrder) {
    const double* th = theta + (long long)kTh * s;
    const int4 gb = gbase[s];
    double wx[4], wz[4][kOrder];
    #pragma unroll
    for (int d = 0; d < 4; ++d) {
      wx[d] = th[(0 * 4 + d) * kOrder + tx];
      #pragma unroll
      for (int t = 0; t < kOrder; ++t) wz[d][t] = th[(2 * 4 + d) * kOrder + t];
    }
    int gx = gb.x - tx;
    if (gx < 0) gx += K;
    double u[4][4];
    #pragma unroll
    for (int a = 0; a < 4; ++a)
      #pragma unroll
      for (int b = 0; b < 4; ++b) u[a][b] = 0.0;
    #pragma unroll
    for (int ty = 0; ty < kOrder; ++ty) {
      double wy[4];
      #pragma unroll
      for (int d = 0; d < 4; ++d) wy[d] = th[(1 * 4 + d) * kOrder + ty];
      int gy = gb.y - ty;
      if (gy < 0) gy += K;
      const long long row = ((long long)gx * K + gy) * K;
      double sz[4] = {0.0, 0.0, 0.0, 0.0};
      #pragma unroll
      for (int tz = 0; tz < kOrder; ++tz) {
        int gz = gb.z - tz;
        if (gz < 0) gz += K;
        const double p = phi[row + gz];
        #pragma unroll
        for (int d = 0; d < 4; ++d) sz[d] += wz[d][tz] * p;
      }
      #pragma unroll
      for (int dy = 0; dy < 4; ++dy)
        #pragma unroll
        for (int dz = 0; dz + dy < 4; ++dz) u[dy][dz] += wy[dy] * sz[dz];
    }
    #pragma unroll
    for (int dx = 0; dx < 4; ++dx)
      #pragma unroll
      for (int dy = 0; dx + dy < 4; ++dy)
        #pragma unroll
        for (int dz = 0; dx + dy + dz < 4; ++dz) v[dx][dy][dz] = wx[dx] * u[dy][dz];
  }
  const unsigned mask = group_mask();
  #pragma unroll
  for (int dx = 0; dx < 4; ++dx)
    #pragma unroll
    for (int dy = 0; dx + dy < 4; ++dy)
      #pragma unroll
      for (int dz = 0; dx + dy + dz < 4; ++dz)
        #pragma unroll
        for (int o = kGroup / 2; o > 0; o >>= 1) v[dx][dy][dz] += __shfl_xor_sync(mask, v[dx][dy][dz], o, kGroup);
  if (tx != 0) return;
  const double4_32a a = A[s], b = B[s], c = C[s], d = D[s];
  const double q = a.w, dp[3] = {b.x, b.y, b.z};
  const double T[3][3] = {{c.x, c.w, d.x}, {c.w, c.y, d.y}, {d.x, d.y, c.z}};
  auto p1 = [&](int a0) {
    int k[3] = {0, 0, 0};
    k[a0]++;
    return v[k[0]][k[1]][k[2]];
  };
  auto p2 = [&](int a0, int a1) {
    int k[3] = {0, 0, 0};
    k[a0]++;
    k[a1]++;
    return v[k[0]][k[1]][k[2]];
  };
  auto p3 = [&](int a0, int a1, int a2) {
    int k[3] = {0, 0, 0};
    k[a0]++;
    k[a1]++;
    k[a2]++;
    return v[k[0]][k[1]][k[2]];
  };
  double* o = out + (long long)kForceAtomStride * s;
  #pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    double f = q * p1(ax);
    #pragma unroll
    for (int bx = 0; bx < 3; ++bx) {
      f += dp[bx] * p2(ax, bx);
      #pragma unroll
      for (int cx = 0; cx < 3; ++cx) f += T[bx][cx] * p3(ax, bx, cx) * (1.0 / 3.0);
    }
    o[ax] = -f;
  }
  o[3] = v[0][0][0];
  o[4] = p1(0);
  o[5] = p1(1);
  o[6] = p1(2);
  o[7] = p2(0, 0) * (1.0 / 3.0);
  o[8] = p2(1, 1) * (1.0 / 3.0);
  o[9] = p2(2, 2) * (1.0 / 3.0);
  o[10] = p2(0, 1) * (2.0 / 3.0);
  o[11] = p2(0, 2) * (2.0 / 3.0);
  o[12] = p2(1, 2) * (2.0 / 3.0);
}

// One block: out = sum_k src[k * stride], k = 0..n-1, in a fixed order.
__global__ void __launch_bounds__(1024) k_block_sum(int n, const double* __restrict__ src, int stride,
                                                    double* __restrict__ out) {
  __shared__ double part[32];
  double s = 0.0;
#pragma unroll 8
  for (int k = threadIdx.x; k < n; k += blockDim.x) s += src[(long long)k * stride];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < (int)(blockDim.x >> 5) ? part[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) *out = s;
  }
}

struct SelfTerms {
  double q, d, th, bg;  // dU/dq = q*q_i + bg*Q_tot, dU/dd = d*d_i, dU/dTheta_ab = th*Theta_ab
};

// Row sums of the per-pair records (double-float, fixed order within each
// lane group) + reciprocal + self + background, times C, quadrupole diagonal
// projected; outputs in caller order; per-atom energy
// 1/2 (q dU/dq + d.dU/dd + Theta.dU/dTheta) in sorted order.
__global__ void __launch_bounds__(256) k_mpole_rows(int n, const int* __restrict__ full_start,
                                                    const int* __restrict__ full_ref, const float2* __restrict__ pair,
                                                    const double* __restrict__ recip,
                                                    const double4_32a* __restrict__ A,
                                                    const double4_32a* __restrict__ B,
                                                    const double4_32a* __restrict__ C,
                                                    const double4_32a* __restrict__ D, const double* __restrict__ qtot,
                                                    SelfTerms st, const int* __restrict__ perm, double* __restrict__ F,
                                                    double* __restrict__ gq, double* __restrict__ gd,
                                                    double* __restrict__ gt, double* __restrict__ e_atom) {
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = gid / kRowGroup, l = gid % kRowGroup;
  if (i >= n) return;
  dflt acc[13];
#pragma unroll
  for (int k = 0; k < 13; ++k) acc[k] = {0.f, 0.f};
  const int e = full_start[i + 1];
  for (int k = full_start[i] + l; k < e; k += kRowGroup) {
    const int ref = full_ref[k];
    const int side = ref & 1;
    // the record is 192 bytes (32-byte aligned): four 32-byte loads take the
    // force (entries 0..2) and this side's derivatives (entries 4..13 or 14..23)
    const float4* p = reinterpret_cast<const float4*>(pair + (long long)kForcePairStride * (ref >> 1));
    float4 w[8];
    ld8_ro(p, w[0], w[1]);
    ld8_ro(p + (side ? 6 : 2), w[2], w[3]);
    ld8_ro(p + (side ? 8 : 4), w[4], w[5]);
    ld8_ro(p + (side ? 10 : 6), w[6], w[7]);
    const float sgn = side ? -1.f : 1.f;
    acc[0] = df_add(acc[0], {sgn * w[0].x, sgn * w[0].y});
    acc[1] = df_add(acc[1], {sgn * w[0].z, sgn * w[0].w});
    acc[2] = df_add(acc[2], {sgn * w[1].x, sgn * w[1].y});
    // w[2..7] hold entries base..base+11 (base = 4 or 12) as (hi, lo) pairs;
    // this side's ten start at entry 4 (side 0) or 14 (side 1)
    float2 v[12];
#pragma unroll
    for (int m = 0; m < 6; ++m) {
      v[2 * m] = make_float2(w[2 + m].x, w[2 + m].y);
      v[2 * m + 1] = make_float2(w[2 + m].z, w[2 + m].w);
    }
#pragma unroll
    for (int m = 0; m < 10; ++m) {
      const float2 x = side ? v[m + 2] : v[m];
      acc[3 + m] = df_add(acc[3 + m], {x.x, x.y});
    }
  }
#pragma unroll
  for (int k = 0; k < 13; ++k) acc[k] = df_group_sum(acc[k]);
  // epilogue spread over the row's lanes: lane l < 13 finishes component l
  // (force x, y, z, q, d x, y, z, Theta xx, yy, zz, xy, xz, yz) in float64
  const double4_32a a = A[i], b = B[i], c = C[i], d = D[i];
  dflt mine = acc[0];
  double m = 0.0, self = 0.0;
#pragma unroll
  for (int k = 1; k < 13; ++k)
    if (l == k) mine = acc[k];
  switch (l) {
    case 3: m = a.w; self = st.q * a.w + st.bg * (*qtot); break;
    case 4: m = b.x; self = st.d * b.x; break;
    case 5: m = b.y; self = st.d * b.y; break;
    case 6: m = b.z; self = st.d * b.z; break;
    case 7: m = c.x; self = st.th * c.x; break;
    case 8: m = c.y; self = st.th * c.y; break;
    case 9: m = c.z; self = st.th * c.z; break;
    case 10: m = c.w; self = 2.0 * st.th * c.w; break;
    case 11: m = d.x; self = 2.0 * st.th * d.x; break;
    case 12: m = d.y; self = 2.0 * st.th * d.y; break;
    default: break;
  }
  const double* rc = recip + (long long)kForceAtomStride * i;
  double v = l < 13 ? (df_to_double(mine) + rc[l] + self) * kCoulomb : 0.0;
  // project the quadrupole diagonal (lanes 7, 8, 9) onto traceless changes
  const unsigned mask = ((1u << kRowGroup) - 1u) << ((threadIdx.x & 31) & ~(kRowGroup - 1));
  const int g0 = (threadIdx.x & 31) & ~(kRowGroup - 1);
  const double mean = (__shfl_sync(mask, v, g0 + 7) + __shfl_sync(mask, v, g0 + 8) + __shfl_sync(mask, v, g0 + 9)) *
                      (1.0 / 3.0);
  if (l >= 7 && l <= 9) v -= mean;
  // per-atom energy 1/2 sum_k moment_k dU/dmoment_k (fixed order over the lanes)
  double u = m * v;
#pragma unroll
  for (int o = kRowGroup / 2; o > 0; o >>= 1) u += __shfl_xor_sync(mask, u, o, kRowGroup);
  if (l == 0) e_atom[i] = 0.5 * u;
  const int o = perm[i];
  if (l < 3) {
    if (F) F[3 * o + l] = v;
  } else if (l == 3) {
    if (gq) gq[o] = v;
  } else if (l < 7) {
    if (gd) gd[3 * o + l - 4] = v;
  } else if (l < 13) {
    if (gt) gt[6 * o + l - 7] = v;
  }
}

dflt split_host(double v) {
  const float h = (float)v;
  return {h, (float)(v - (double)h)};
}

}  // namespace

int multipole_energy(amp_ctx* c, double* U, double* F, double* gq, double* gd, double* gt) {
  int r;
  if (c->mpole_e_cap < c->n_cap) {
    dev_free(c, c->mpole_e);
    c->mpole_e = nullptr;
    if ((r = dev_alloc(c, &c->mpole_e, c->n_cap))) return r;
    c->mpole_e_cap = c->n_cap;
  }
  cudaStream_t s = c->stream;
  if (c->cluster) {
    PhaseScope ps(c, AMP_PHASE_FORCES);
    launch_split_multipoles(c);
    c->n_launch += 2;
    k_mpole_cluster_df<<<amp_blocks(c->n, 128), 128, 0, s>>>(c->n, c->pd, c->mp_df, c->atomA, c->atomB, c->atomC,
                                                            c->atomD, c->perm, F, gq, gd, gt, c->mpole_e);
    k_block_sum<<<1, 1024, 0, s>>>(c->n, c->mpole_e, 1, c->scal + 5);
  } else {
    pme_theta64(c, c->stream);
    if ((r = force_buffers(c))) return r;
    const double b = c->cfg.ewald_beta, L = c->cfg.box;
    MGeomDf g;
    g.L = split_host(L);
    g.beta = split_host(b);
    g.twob2 = split_host(2.0 * b * b);
    g.gpre = split_host(2.0 * b / kSqrtPi);
    g.invL = (float)(1.0 / L);
    const double c0 = 2.0 * b / kSqrtPi;
    SelfTerms st;
    st.q = -c0;
    st.d = -c0 * (2.0 * b * b / 3.0);
    st.th = -c0 * (8.0 * b * b * b * b / 45.0);
    st.bg = -3.14159265358979323846 / (L * L * L * b * b);
    // the per-pair records are (hi, lo) float pairs in the backward pair buffer
    float2* pair = reinterpret_cast<float2*>(c->force_pair);
    PhaseScope ps(c, AMP_PHASE_FORCES);
    if ((r = pme_potential(c, false, true, nullptr, nullptr, c->grid64b, c->stream))) return r;
    c->n_launch += 2;
    k_recip_mpole<<<amp_blocks((long long)c->n * kGroup, 128), 128, 0, s>>>(
        c->n, c->theta, c->gbase, c->grid64b, c->K, c->atomA, c->atomB, c->atomC, c->atomD, c->force_recip);
    k_block_sum<<<1, 1024, 0, s>>>(c->n, reinterpret_cast<const double*>(c->atomA) + 3, 4, c->scal + 4);
    if (c->n_half > 0) {
      c->n_launch += 1;
      k_mpole_pairs_df<<<amp_blocks(c->n_half, 128), 128, 0, s>>>(c->n_half, c->half_i, c->half_j, c->pd,
                                                                   c->mp_df, g, c->dfm, pair);
    }
    c->n_launch += 2;
    k_mpole_rows<<<amp_blocks((long long)c->n * kRowGroup, 256), 256, 0, s>>>(
        c->n, c->full_start, c->full_ref, pair, c->force_recip, c->atomA, c->atomB, c->atomC, c->atomD,
        c->scal + 4, st, c->perm, F, gq, gd, gt, c->mpole_e);
    k_block_sum<<<1, 1024, 0, s>>>(c->n, c->mpole_e, 1, c->scal + 5);
  }
  if ((r = cuda_check(c, cudaGetLastError(), "multipole energy launch"))) return r;
  if (!U) return AMP_OK;
  cudaMemcpyAsync(c->hbuf + 5, c->scal + 5, sizeof(double), cudaMemcpyDeviceToHost, s);
  if ((r = cuda_check(c, cudaStreamSynchronize(s), "multipole energy"))) return r;
  *U = c->hbuf[5];
  return AMP_OK;
}

}  // namespace amp
