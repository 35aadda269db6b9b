// Adjoint backward: polarization forces and multipole-moment gradients
// (kernel for the "epolar1" forces of the paper's Section "Hotspots").
//
// The energy U = C (1/2 mu.A mu - mu.E0) is stationary in mu at the solution,
// so every gradient is taken at fixed mu (no re-solve):
//   F_k = C [1/2 d(mu.T mu)/dr_k + d(mu.E0)/dr_k],
//   dU/d(moment) = -C d(mu.E0)/d(moment).
// Real space, unique pair (i, j), r = x_i - x_j, damped kernels
//   B_n^eff = B_n - (1 - s l_{2n+1}) bare_n,
//   dB_n^eff/dr = -r B_{n+1} + s l' bare_n + (1 - s l) r bare_{n+1},
//   l3' = 3x/r e^-x, l5' = 3x^2/r e^-x, l7' = 3x/r (0.6 x^2 - 0.2 x) e^-x:
//   mutual: grad W = [-B1u'(mu_i.mu_j) + B2u'(mu_i.r)(mu_j.r)] r/|r|
//                    + B2u [mu_i (mu_j.r) + mu_j (mu_i.r)];
//   permanent: grad_r (mu.E) of a dipole in a multipole's field (see below).
// One thread per unique pair writes its force and both ends' moment gradients
// to a per-pair buffer; one group of lanes per atom sums its row in a fixed
// order (no atomics). Reciprocal space: phi_mu = conv(spread mu), phi_M =
// conv(spread q, d, Theta); per atom the interpolated derivatives up to third
// order (8-lane groups, one lane per x plane) give
//   F_a = -C [sum_b mu_b (phi_M,ab + phi_mu,ab) + q phi_mu,a + sum_b d_b phi_mu,ab
//             + 1/3 sum_bc Theta_bc phi_mu,abc],
//   dU/dq = C phi_mu, dU/dd = C grad phi_mu, dU/dTheta_ab = C/3 phi_mu,ab (x2 off-diagonal);
// self term dU/dd_k -= C 4 beta^3/(3 sqrt(pi)) mu_k.
#include "amp_internal.cuh"

namespace amp {
namespace {

constexpr int kPairStride = kForcePairStride;   // force(3), pad, side0 grads(10), side1 grads(10)
constexpr int kRecipStride = kForceAtomStride;  // force(3), gq, gd(3), gquad(6), pad(3)
constexpr int kTh = 3 * 4 * kOrder;
constexpr int kGroup = 8;

struct FGeom {
  double L, beta, twob2, gpre, selfc;
};

__device__ __forceinline__ double min_image(double d, double L) { return d - L * rint(d / L); }

template <typename R>
struct V3 {
  R x, y, z;
};

template <typename R>
__device__ __forceinline__ R dot(const V3<R>& a, const V3<R>& b) {
  return a.x * b.x + a.y * b.y + a.z * b.z;
}

// Theta (xx,yy,zz,xy,xz,yz) times v
template <typename R>
__device__ __forceinline__ V3<R> th_mul(const R* t, const V3<R>& v) {
  return {t[0] * v.x + t[3] * v.y + t[4] * v.z, t[3] * v.x + t[1] * v.y + t[5] * v.z,
          t[4] * v.x + t[5] * v.y + t[2] * v.z};
}

// grad_r (mu . E(r)) for the field of a multipole (q, d, Theta) at displacement r
template <typename R>
__device__ __forceinline__ V3<R> grad_mu_field(const V3<R>& r, R ir, const V3<R>& mu, R q, const V3<R>& d,
                                               const R* th, R b1, R b2, R b3, R db1, R db2, R db3) {
  const V3<R> thr = th_mul(th, r), thmu = th_mul(th, mu);
  const R rthr = dot(r, thr), mr = dot(mu, r), dr = dot(d, r), md = dot(mu, d), mthr = dot(mu, thr);
  const R radial = (db1 * (q * mr - md) + db2 * (dr * mr - (R)(2.0 / 3.0) * mthr) + db3 * rthr * mr * (R)(1.0 / 3.0)) * ir;
  const R c2 = (R)(2.0 / 3.0) * b2, c3 = b3 * (R)(1.0 / 3.0);
  V3<R> g;
  g.x = radial * r.x + q * b1 * mu.x + b2 * (d.x * mr + mu.x * dr) - c2 * thmu.x + c3 * ((R)2 * thr.x * mr + rthr * mu.x);
  g.y = radial * r.y + q * b1 * mu.y + b2 * (d.y * mr + mu.y * dr) - c2 * thmu.y + c3 * ((R)2 * thr.y * mr + rthr * mu.y);
  g.z = radial * r.z + q * b1 * mu.z + b2 * (d.z * mr + mu.z * dr) - c2 * thmu.z + c3 * ((R)2 * thr.z * mr + rthr * mu.z);
  return g;
}

// d(mu.E)/d(q, d, Theta6) of the source at displacement r, times `scale`, into o[10]
template <typename R>
__device__ __forceinline__ void moment_grads(const V3<R>& r, const V3<R>& mu, R b1, R b2, R b3, double scale,
                                             double* o) {
  const R mr = dot(mu, r);
  const R c2 = (R)(2.0 / 3.0) * b2, c3 = b3 * mr * (R)(1.0 / 3.0);
  o[0] = scale * (double)(b1 * mr);
  o[1] = scale * (double)(-b1 * mu.x + b2 * mr * r.x);
  o[2] = scale * (double)(-b1 * mu.y + b2 * mr * r.y);
  o[3] = scale * (double)(-b1 * mu.z + b2 * mr * r.z);
  o[4] = scale * (double)(-c2 * mu.x * r.x + c3 * r.x * r.x);
  o[5] = scale * (double)(-c2 * mu.y * r.y + c3 * r.y * r.y);
  o[6] = scale * (double)(-c2 * mu.z * r.z + c3 * r.z * r.z);
  o[7] = scale * (double)(-c2 * (mu.x * r.y + mu.y * r.x) + (R)2 * c3 * r.x * r.y);
  o[8] = scale * (double)(-c2 * (mu.x * r.z + mu.z * r.x) + (R)2 * c3 * r.x * r.z);
  o[9] = scale * (double)(-c2 * (mu.y * r.z + mu.z * r.y) + (R)2 * c3 * r.y * r.z);
}

// Bilinear mode (TCG-1 gradients): the field vector c (in place of mu)
// enters with weight sf, and the operator part is the gradient of
// a1.T b1 + a2.T b2 (both orderings of each pair) instead of 1/2 mu.T mu:
//   F_pair = C [sf (g1 - g2) + sum_k (gw(a_k,i, b_k,j) + gw(a_k,j, b_k,i))],
//   moments: -C sf d(c.E)/d(moment).
struct Bilinear {
  const double4_32a *a1, *b1, *a2, *b2;
  double sf;
};

template <typename R>
__device__ __forceinline__ V3<R> grad_w(const V3<R>& r, R ir, const V3<R>& x, const V3<R>& y, R b2u, R db1u,
                                        R db2u) {  // grad_r of x.T(r) y = -B1u x.y + B2u (x.r)(y.r)
  const R xy = dot(x, y), xr = dot(x, r), yr = dot(y, r);
  const R rad = (-db1u * xy + db2u * xr * yr) * ir;
  return {rad * r.x + b2u * (x.x * yr + y.x * xr), rad * r.y + b2u * (x.y * yr + y.y * xr),
          rad * r.z + b2u * (x.z * yr + y.z * xr)};
}

template <typename R>
__device__ __forceinline__ V3<R> v3(const double4_32a& v) {
  return {(R)v.x, (R)v.y, (R)v.z};
}

template <typename R, bool kBil>
__global__ void __launch_bounds__(256) k_pair_forces(long long nh, const int* __restrict__ half_i,
                                                     const int* __restrict__ half_j,
                                                     const double4_32a* __restrict__ A,
                                                     const double4_32a* __restrict__ B,
                                                     const double4_32a* __restrict__ C,
                                                     const double4_32a* __restrict__ D,
                                                     const double4_32a* __restrict__ mu, FGeom g, Bilinear bl,
                                                     double* __restrict__ out) {
  const long long pid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (pid >= nh) return;
  const int i = half_i[pid], j = half_j[pid];
  const double4_32a ai = A[i], aj = A[j], bi = B[i], bj = B[j], ci = C[i], cj = C[j], di = D[i], dj = D[j];
  const double4_32a mi4 = mu[i], mj4 = mu[j];
  const V3<R> r = {(R)min_image(ai.x - aj.x, g.L), (R)min_image(ai.y - aj.y, g.L), (R)min_image(ai.z - aj.z, g.L)};
  const V3<R> nr = {-r.x, -r.y, -r.z};
  const R r2 = dot(r, r);
  const R rr = sqrt(r2);
  const R ir = (R)1 / rr, ir2 = ir * ir;
  const R beta = (R)g.beta, br = beta * rr;
  R fac = exp(-br * br) * (R)g.gpre;
  const R tb2 = (R)g.twob2;
  const R B0 = erfc(br) * ir;
  const R B1 = (B0 + fac) * ir2;
  fac *= tb2;
  const R B2 = ((R)3 * B1 + fac) * ir2;
  fac *= tb2;
  const R B3 = ((R)5 * B2 + fac) * ir2;
  fac *= tb2;
  const R B4 = ((R)7 * B3 + fac) * ir2;
  const R e1 = ir * ir2, e2 = (R)3 * e1 * ir2, e3 = (R)5 * e2 * ir2, e4 = (R)7 * e3 * ir2;  // bare
  const R x = min((R)di.z, (R)dj.z) * r2 * rr * (R)bi.w * (R)bj.w;
  const R e = exp(-x);
  const R dxdr = (R)3 * x * ir;
  const R o3 = e, o5 = ((R)1 + x) * e, o7 = ((R)1 + x + (R)0.6 * x * x) * e;
  const R l3p = dxdr * e, l5p = dxdr * x * e, l7p = dxdr * ((R)0.6 * x * x - (R)0.2 * x) * e;
  // mutual kernels (every pair damped)
  const R b1u = B1 - o3 * e1, db1u = -rr * B2 + l3p * e1 + o3 * rr * e2;
  const R b2u = B2 - o5 * e2, db2u = -rr * B3 + l5p * e2 + o5 * rr * e3;
  // permanent kernels (exclusion inside a molecule)
  R b1, b2, b3, db1, db2, db3;
  if (di.w == dj.w) {
    b1 = B1 - e1;
    b2 = B2 - e2;
    b3 = B3 - e3;
    db1 = -rr * B2 + rr * e2;
    db2 = -rr * B3 + rr * e3;
    db3 = -rr * B4 + rr * e4;
  } else {
    b1 = b1u;
    b2 = b2u;
    db1 = db1u;
    db2 = db2u;
    b3 = B3 - o7 * e3;
    db3 = -rr * B4 + l7p * e3 + o7 * rr * e4;
  }
  const V3<R> mi = {(R)mi4.x, (R)mi4.y, (R)mi4.z}, mj = {(R)mj4.x, (R)mj4.y, (R)mj4.z};
  V3<R> gw;
  R sf = (R)1;
  if (kBil) {
    sf = (R)bl.sf;
    const V3<R> w1 = grad_w<R>(r, ir, v3<R>(bl.a1[i]), v3<R>(bl.b1[j]), b2u, db1u, db2u);
    const V3<R> w2 = grad_w<R>(r, ir, v3<R>(bl.a1[j]), v3<R>(bl.b1[i]), b2u, db1u, db2u);
    gw = {w1.x + w2.x, w1.y + w2.y, w1.z + w2.z};
    if (bl.a2) {
      const V3<R> w3 = grad_w<R>(r, ir, v3<R>(bl.a2[i]), v3<R>(bl.b2[j]), b2u, db1u, db2u);
      const V3<R> w4 = grad_w<R>(r, ir, v3<R>(bl.a2[j]), v3<R>(bl.b2[i]), b2u, db1u, db2u);
      gw = {gw.x + w3.x + w4.x, gw.y + w3.y + w4.y, gw.z + w3.z + w4.z};
    }
  } else {
    gw = grad_w<R>(r, ir, mi, mj, b2u, db1u, db2u);
  }
  const R thi[6] = {(R)ci.x, (R)ci.y, (R)ci.z, (R)ci.w, (R)di.x, (R)di.y};
  const R thj[6] = {(R)cj.x, (R)cj.y, (R)cj.z, (R)cj.w, (R)dj.x, (R)dj.y};
  const V3<R> dpi = {(R)bi.x, (R)bi.y, (R)bi.z}, dpj = {(R)bj.x, (R)bj.y, (R)bj.z};
  const V3<R> g1 = grad_mu_field<R>(r, ir, mi, (R)aj.w, dpj, thj, b1, b2, b3, db1, db2, db3);
  const V3<R> g2 = grad_mu_field<R>(nr, ir, mj, (R)ai.w, dpi, thi, b1, b2, b3, db1, db2, db3);
  double* o = out + kPairStride * pid;
  o[0] = kCoulomb * (double)(gw.x + sf * (g1.x - g2.x));
  o[1] = kCoulomb * (double)(gw.y + sf * (g1.y - g2.y));
  o[2] = kCoulomb * (double)(gw.z + sf * (g1.z - g2.z));
  o[3] = 0.0;
  const double ms = -kCoulomb * (kBil ? bl.sf : 1.0);
  moment_grads<R>(nr, mj, b1, b2, b3, ms, o + 4);   // owner i's moments, seen by mu_j
  moment_grads<R>(r, mi, b1, b2, b3, ms, o + 14);   // j's moments, seen by mu_i
}

// The two-field form's extra term 1/2 C d(mu_d . (E_p - E_d)) for the
// intramolecular pairs (E_p - E_d: their Thole-damped bare fields times s),
// added to the per-pair records of k_pair_forces: kernels b_n = s l bare_n,
// db_n/dr = s (l' bare_n - l r bare_{n+1}).
__global__ void __launch_bounds__(128) k_intra_pair_grads(const int* __restrict__ intra,
                                                          const int* __restrict__ half_i,
                                                          const int* __restrict__ half_j,
                                                          const double4_32a* __restrict__ A,
                                                          const double4_32a* __restrict__ B,
                                                          const double4_32a* __restrict__ C,
                                                          const double4_32a* __restrict__ D,
                                                          const double4_32a* __restrict__ mu, FGeom g, double s,
                                                          double* __restrict__ out) {
  const int cnt = intra[0];
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < cnt; k += gridDim.x * blockDim.x) {
    const int pid = intra[1 + k];
    const int i = half_i[pid], j = half_j[pid];
    const double4_32a ai = A[i], aj = A[j], bi = B[i], bj = B[j], ci = C[i], cj = C[j], di = D[i], dj = D[j];
    const V3<double> r = {min_image(ai.x - aj.x, g.L), min_image(ai.y - aj.y, g.L), min_image(ai.z - aj.z, g.L)};
    const V3<double> nr = {-r.x, -r.y, -r.z};
    const double r2 = dot(r, r), rr = sqrt(r2), ir = 1.0 / rr, ir2 = ir * ir;
    const double e1 = ir * ir2, e2 = 3.0 * e1 * ir2, e3 = 5.0 * e2 * ir2, e4 = 7.0 * e3 * ir2;
    const double x = fmin(di.z, dj.z) * r2 * rr * bi.w * bj.w;
    const double e = exp(-x), dxdr = 3.0 * x * ir;
    const double l3 = 1.0 - e, l5 = 1.0 - (1.0 + x) * e, l7 = 1.0 - (1.0 + x + 0.6 * x * x) * e;
    const double l3p = dxdr * e, l5p = dxdr * x * e, l7p = dxdr * (0.6 * x * x - 0.2 * x) * e;
    const double b1 = s * l3 * e1, b2 = s * l5 * e2, b3 = s * l7 * e3;
    const double db1 = s * (l3p * e1 - l3 * rr * e2), db2 = s * (l5p * e2 - l5 * rr * e3),
                 db3 = s * (l7p * e3 - l7 * rr * e4);
    const V3<double> mi = {mu[i].x, mu[i].y, mu[i].z}, mj = {mu[j].x, mu[j].y, mu[j].z};
    const double thi[6] = {ci.x, ci.y, ci.z, ci.w, di.x, di.y};
    const double thj[6] = {cj.x, cj.y, cj.z, cj.w, dj.x, dj.y};
    const V3<double> dpi = {bi.x, bi.y, bi.z}, dpj = {bj.x, bj.y, bj.z};
    const V3<double> g1 = grad_mu_field<double>(r, ir, mi, aj.w, dpj, thj, b1, b2, b3, db1, db2, db3);
    const V3<double> g2 = grad_mu_field<double>(nr, ir, mj, ai.w, dpi, thi, b1, b2, b3, db1, db2, db3);
    double* o = out + kPairStride * (long long)pid;
    o[0] += 0.5 * kCoulomb * (g1.x - g2.x);
    o[1] += 0.5 * kCoulomb * (g1.y - g2.y);
    o[2] += 0.5 * kCoulomb * (g1.z - g2.z);
    double m[10];
    moment_grads<double>(nr, mj, b1, b2, b3, -0.5 * kCoulomb, m);
    for (int t = 0; t < 10; ++t) o[4 + t] += m[t];
    moment_grads<double>(r, mi, b1, b2, b3, -0.5 * kCoulomb, m);
    for (int t = 0; t < 10; ++t) o[14 + t] += m[t];
  }
}

__device__ __forceinline__ unsigned group_mask() {
  return ((1u << kGroup) - 1u) << ((threadIdx.x & 31) & ~(kGroup - 1));
}

// Reciprocal gradients: interpolated derivatives of phi_mu (orders 0..3) and
// phi_M (order 2) at every atom, then the force and moment gradients.
template <typename R>
__global__ void __launch_bounds__(128) k_recip_gradients(int n, const R* __restrict__ theta,
                                                         const int4* __restrict__ gbase,
                                                         const R* __restrict__ phi_mu, const R* __restrict__ phi_m,
                                                         int K, const double4_32a* __restrict__ mu,
                                                         const double4_32a* __restrict__ A,
                                                         const double4_32a* __restrict__ B,
                                                         const double4_32a* __restrict__ C,
                                                         const double4_32a* __restrict__ D, double sf,
                                                         double wq, double* __restrict__ recip) {
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  const int s = gid / kGroup, tx = gid % kGroup;
  if (s >= n) return;
  // v[dx][dy][dz] for dx+dy+dz <= 3 (phi_mu) and m[dx][dy][dz] for sum == 2 (phi_M)
  double v[4][4][4], m[3][3][3];
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b)
      for (int c = 0; c < 4; ++c) v[a][b][c] = 0.0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      for (int c = 0; c < 3; ++c) m[a][b][c] = 0.0;
  const int4 gb = gbase[s];
  if (tx < kOrder) {
    const R* th = theta + (long long)kTh * s;
    R wx[4], wz[4][kOrder];
    for (int d = 0; d < 4; ++d) {
      wx[d] = th[(0 * 4 + d) * kOrder + tx];
      for (int t = 0; t < kOrder; ++t) wz[d][t] = th[(2 * 4 + d) * kOrder + t];
    }
    int gx = gb.x - tx;
    if (gx < 0) gx += K;
    R u[4][4], um[3][3];
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) u[a][b] = 0;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) um[a][b] = 0;
    for (int ty = 0; ty < kOrder; ++ty) {
      R wy[4];
      for (int d = 0; d < 4; ++d) wy[d] = th[(1 * 4 + d) * kOrder + ty];
      int gy = gb.y - ty;
      if (gy < 0) gy += K;
      const long long row = ((long long)gx * K + gy) * K;
      R sz[4] = {0, 0, 0, 0}, smz[3] = {0, 0, 0};
      for (int tz = 0; tz < kOrder; ++tz) {
        int gz = gb.z - tz;
        if (gz < 0) gz += K;
        const R p = phi_mu[row + gz], pm = phi_m[row + gz];
        for (int d = 0; d < 4; ++d) sz[d] += wz[d][tz] * p;
        for (int d = 0; d < 3; ++d) smz[d] += wz[d][tz] * pm;
      }
      for (int dy = 0; dy < 4; ++dy)
        for (int dz = 0; dz + dy < 4; ++dz) u[dy][dz] += wy[dy] * sz[dz];
      for (int dy = 0; dy < 3; ++dy)
        for (int dz = 0; dz + dy < 3; ++dz) um[dy][dz] += wy[dy] * smz[dz];
    }
    for (int dx = 0; dx < 4; ++dx)
      for (int dy = 0; dx + dy < 4; ++dy)
        for (int dz = 0; dx + dy + dz < 4; ++dz) v[dx][dy][dz] = (double)(wx[dx] * u[dy][dz]);
    for (int dx = 0; dx < 3; ++dx)
      for (int dy = 0; dx + dy < 3; ++dy) {
        const int dz = 2 - dx - dy;
        m[dx][dy][dz] = (double)(wx[dx] * um[dy][dz]);
      }
  }
  const unsigned mask = group_mask();
  for (int dx = 0; dx < 4; ++dx)
    for (int dy = 0; dx + dy < 4; ++dy)
      for (int dz = 0; dx + dy + dz < 4; ++dz)
        for (int o = kGroup / 2; o > 0; o >>= 1) v[dx][dy][dz] += __shfl_xor_sync(mask, v[dx][dy][dz], o, kGroup);
  for (int dx = 0; dx < 3; ++dx)
    for (int dy = 0; dx + dy < 3; ++dy) {
      const int dz = 2 - dx - dy;
      for (int o = kGroup / 2; o > 0; o >>= 1) m[dx][dy][dz] += __shfl_xor_sync(mask, m[dx][dy][dz], o, kGroup);
    }
  if (tx != 0) return;
  const double4_32a a = A[s], b = B[s], c = C[s], d = D[s], mm = mu[s];
  const double q = a.w, dp[3] = {b.x, b.y, b.z}, m3[3] = {mm.x, mm.y, mm.z};
  const double T[3][3] = {{c.x, c.w, d.x}, {c.w, c.y, d.y}, {d.x, d.y, c.z}};
  // derivative accessors by axis list
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
  auto m2 = [&](int a0, int a1) {
    int k[3] = {0, 0, 0};
    k[a0]++;
    k[a1]++;
    return m[k[0]][k[1]][k[2]];
  };
  auto p3 = [&](int a0, int a1, int a2) {
    int k[3] = {0, 0, 0};
    k[a0]++;
    k[a1]++;
    k[a2]++;
    return v[k[0]][k[1]][k[2]];
  };
  // sf: weight of c.E (field points and sources moving); wq: of the
  // quadratic 1/2 c.T c (1 for the polarization forces, 0 in bilinear mode)
  double* out = recip + (long long)kRecipStride * s;
  for (int ax = 0; ax < 3; ++ax) {
    double f = q * p1(ax), fq = 0.0;
    for (int bx = 0; bx < 3; ++bx) {
      f += m3[bx] * m2(ax, bx) + dp[bx] * p2(ax, bx);
      fq += m3[bx] * p2(ax, bx);
      for (int cx = 0; cx < 3; ++cx) f += T[bx][cx] * p3(ax, bx, cx) * (1.0 / 3.0);
    }
    out[ax] = -kCoulomb * (sf * f + wq * fq);
  }
  const double cs = kCoulomb * sf;
  out[3] = cs * v[0][0][0];
  out[4] = cs * p1(0);
  out[5] = cs * p1(1);
  out[6] = cs * p1(2);
  out[7] = cs * p2(0, 0) / 3.0;
  out[8] = cs * p2(1, 1) / 3.0;
  out[9] = cs * p2(2, 2) / 3.0;
  out[10] = cs * 2.0 * p2(0, 1) / 3.0;
  out[11] = cs * 2.0 * p2(0, 2) / 3.0;
  out[12] = cs * 2.0 * p2(1, 2) / 3.0;
}

// Reciprocal part of bilinear forms: F -= C y.H_x at every atom, H_x the
// interpolated second derivatives of the grid potential phi_x of the dipoles
// x (d(a.T_rec b)/dr_k = -(a_k.H_b + b_k.H_a): each spread moves with its
// atom). Same lane layout as k_recip_gradients; adds to recip[s][0..2].
template <typename R>
__global__ void __launch_bounds__(128) k_recip_hessian_dot(int n, const R* __restrict__ theta,
                                                           const int4* __restrict__ gbase,
                                                           const R* __restrict__ phi_x, int K,
                                                           const double4_32a* __restrict__ y,
                                                           double* __restrict__ recip) {
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  const int s = gid / kGroup, tx = gid % kGroup;
  if (s >= n) return;
  double h[3][3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      for (int c = 0; c < 3; ++c) h[a][b][c] = 0.0;
  const int4 gb = gbase[s];
  if (tx < kOrder) {
    const R* th = theta + (long long)kTh * s;
    R wx[3], wz[3][kOrder];
    for (int d = 0; d < 3; ++d) {
      wx[d] = th[(0 * 4 + d) * kOrder + tx];
      for (int t = 0; t < kOrder; ++t) wz[d][t] = th[(2 * 4 + d) * kOrder + t];
    }
    int gx = gb.x - tx;
    if (gx < 0) gx += K;
    R u[3][3];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) u[a][b] = 0;
    for (int ty = 0; ty < kOrder; ++ty) {
      R wy[3];
      for (int d = 0; d < 3; ++d) wy[d] = th[(1 * 4 + d) * kOrder + ty];
      int gy = gb.y - ty;
      if (gy < 0) gy += K;
      const long long row = ((long long)gx * K + gy) * K;
      R sz[3] = {0, 0, 0};
      for (int tz = 0; tz < kOrder; ++tz) {
        int gz = gb.z - tz;
        if (gz < 0) gz += K;
        const R p = phi_x[row + gz];
        for (int d = 0; d < 3; ++d) sz[d] += wz[d][tz] * p;
      }
      for (int dy = 0; dy < 3; ++dy)
        for (int dz = 0; dz + dy < 3; ++dz) u[dy][dz] += wy[dy] * sz[dz];
    }
    for (int dx = 0; dx < 3; ++dx)
      for (int dy = 0; dx + dy < 3; ++dy) {
        const int dz = 2 - dx - dy;
        h[dx][dy][dz] = (double)(wx[dx] * u[dy][dz]);
      }
  }
  const unsigned mask = group_mask();
  for (int dx = 0; dx < 3; ++dx)
    for (int dy = 0; dx + dy < 3; ++dy) {
      const int dz = 2 - dx - dy;
      for (int o = kGroup / 2; o > 0; o >>= 1) h[dx][dy][dz] += __shfl_xor_sync(mask, h[dx][dy][dz], o, kGroup);
    }
  if (tx != 0) return;
  const double4_32a yy = y[s];
  const double yv[3] = {yy.x, yy.y, yy.z};
  double* out = recip + (long long)kRecipStride * s;
  for (int ax = 0; ax < 3; ++ax) {
    double f = 0.0;
    for (int bx = 0; bx < 3; ++bx) {
      int k[3] = {0, 0, 0};
      k[ax]++;
      k[bx]++;
      f += yv[bx] * h[k[0]][k[1]][k[2]];
    }
    out[ax] -= kCoulomb * f;
  }
}

__device__ __forceinline__ double gsum(double v) {
  const unsigned mask = ((1u << kRowGroup) - 1u) << ((threadIdx.x & 31) & ~(kRowGroup - 1));
#pragma unroll
  for (int o = kRowGroup / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o, kRowGroup);
  return v;
}

// Row sums of the per-pair terms + reciprocal + self, written in caller order.
__global__ void __launch_bounds__(256) k_force_rows(int n, const int* __restrict__ full_start,
                                                    const int* __restrict__ full_ref, const double* __restrict__ pair,
                                                    const double* __restrict__ recip, const double4_32a* __restrict__ mu,
                                                    double selfc, const int* __restrict__ perm, double* __restrict__ F,
                                                    double* __restrict__ gq, double* __restrict__ gd,
                                                    double* __restrict__ gt) {
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = gid / kRowGroup, l = gid % kRowGroup;
  if (i >= n) return;
  double acc[13];
  for (int k = 0; k < 13; ++k) acc[k] = 0.0;
  const int e = full_start[i + 1];
  for (int k = full_start[i] + l; k < e; k += kRowGroup) {
    const int ref = full_ref[k];
    const double* p = pair + (long long)kPairStride * (ref >> 1);
    const double sgn = (ref & 1) ? -1.0 : 1.0;
    acc[0] += sgn * p[0];
    acc[1] += sgn * p[1];
    acc[2] += sgn * p[2];
    const double* g = p + 4 + 10 * (ref & 1);
    for (int m = 0; m < 10; ++m) acc[3 + m] += g[m];
  }
  for (int k = 0; k < 13; ++k) acc[k] = gsum(acc[k]);
  if (l != 0) return;
  const int o = perm[i];
  if (recip)
    for (int k = 0; k < 13; ++k) acc[k] += recip[(long long)kRecipStride * i + k];
  const double4_32a m = mu[i];
  acc[4] -= kCoulomb * selfc * m.x;
  acc[5] -= kCoulomb * selfc * m.y;
  acc[6] -= kCoulomb * selfc * m.z;
  F[3 * o] = acc[0];
  F[3 * o + 1] = acc[1];
  F[3 * o + 2] = acc[2];
  if (gq) gq[o] = acc[3];
  if (gd) {
    gd[3 * o] = acc[4];
    gd[3 * o + 1] = acc[5];
    gd[3 * o + 2] = acc[6];
  }
  if (gt)
    for (int k = 0; k < 6; ++k) gt[6 * o + k] = acc[7 + k];
}

__global__ void k_two_rhs_vectors(int n, const double4_32a* __restrict__ mu_d, const double4_32a* __restrict__ mu_p,
                                  double4_32a* __restrict__ csum, double4_32a* __restrict__ half_p) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double4_32a d = mu_d[k], p = mu_p[k];
  csum[k] = make_double4_32a(d.x + p.x, d.y + p.y, d.z + p.z, 0.0);
  half_p[k] = make_double4_32a(0.5 * p.x, 0.5 * p.y, 0.5 * p.z, 0.0);
}

}  // namespace

// Per-pair (24 doubles) and per-atom (16 doubles) backward buffers, sized
// with the lists, and the second float64 grid.
int force_buffers(amp_ctx* c) {
  int r;
  if (c->force_pair_cap < c->cap_half) {
    dev_free(c, c->force_pair);
    c->force_pair = nullptr;
    if ((r = dev_alloc(c, &c->force_pair, kPairStride * c->cap_half))) return r;
    c->force_pair_cap = c->cap_half;
  }
  if (c->force_atom_cap < c->n_cap) {
    dev_free(c, c->force_recip);
    c->force_recip = nullptr;
    if ((r = dev_alloc(c, &c->force_recip, (long long)kRecipStride * c->n_cap))) return r;
    c->force_atom_cap = c->n_cap;
  }
  const long long ng = (long long)c->K * c->K * c->K;
  if (!c->grid64b && (r = dev_alloc(c, &c->grid64b, ng))) return r;
  return AMP_OK;
}

int forces(amp_ctx* c, const double4_32a* mu_sorted, double* F, double* gq, double* gd, double* gt) {
  const bool fp32 = c->cfg.precision == AMP_MIXED;
  int r;
  pme_theta64(c, c->stream);  // the float64 B-spline weights (float64 path: built on first use)
  if ((r = force_buffers(c))) return r;
  const long long ng = (long long)c->K * c->K * c->K;
  if (fp32 && !c->grid32b && (r = dev_alloc(c, &c->grid32b, ng))) return r;
  FGeom g;
  const double b = c->cfg.ewald_beta;
  g.L = c->cfg.box;
  g.beta = b;
  g.twob2 = 2.0 * b * b;
  g.gpre = 2.0 * b * b / (b * kSqrtPi);
  g.selfc = 4.0 * b * b * b / (3.0 * kSqrtPi);
  cudaStream_t st = c->stream;
  {
    PhaseScope ps(c, AMP_PHASE_FORCES);
    // reciprocal: phi_mu into the primary grid, phi_M into the second grid
    if (fp32) {
      launch_to32(c, mu_sorted, c->p32);
      if ((r = pme_potential(c, true, false, mu_sorted, c->p32, c->grid32, c->stream))) return r;
      if ((r = pme_potential(c, true, true, nullptr, nullptr, c->grid32b, c->stream))) return r;
      c->n_launch += 1;
      k_recip_gradients<float><<<amp_blocks((long long)c->n * kGroup, 128), 128, 0, st>>>(
          c->n, c->theta32, c->gbase, c->grid32, c->grid32b, c->K, mu_sorted, c->atomA, c->atomB, c->atomC,
          c->atomD, 1.0, 1.0, c->force_recip);
    } else {
      if ((r = pme_potential(c, false, false, mu_sorted, nullptr, c->grid64, c->stream))) return r;
      if ((r = pme_potential(c, false, true, nullptr, nullptr, c->grid64b, c->stream))) return r;
      c->n_launch += 1;
      k_recip_gradients<double><<<amp_blocks((long long)c->n * kGroup, 128), 128, 0, st>>>(
          c->n, c->theta, c->gbase, c->grid64, c->grid64b, c->K, mu_sorted, c->atomA, c->atomB, c->atomC,
          c->atomD, 1.0, 1.0, c->force_recip);
    }
    if (c->n_half > 0) {
      c->n_launch += 1;
      const Bilinear none{nullptr, nullptr, nullptr, nullptr, 1.0};
      if (fp32)
        k_pair_forces<float, false><<<amp_blocks(c->n_half, 256), 256, 0, st>>>(
            c->n_half, c->half_i, c->half_j, c->atomA, c->atomB, c->atomC, c->atomD, mu_sorted, g, none,
            c->force_pair);
      else
        k_pair_forces<double, false><<<amp_blocks(c->n_half, 256), 256, 0, st>>>(
            c->n_half, c->half_i, c->half_j, c->atomA, c->atomB, c->atomC, c->atomD, mu_sorted, g, none,
            c->force_pair);
    }
    c->n_launch += 1;
    k_force_rows<<<amp_blocks((long long)c->n * kRowGroup, 256), 256, 0, st>>>(
        c->n, c->full_start, c->full_ref, c->force_pair, c->force_recip, mu_sorted, g.selfc, c->perm, F, gq, gd, gt);
  }
  return cuda_check(c, cudaGetLastError(), "forces launch");
}

// Gradients of sf c.E + a1.T b1 + a2.T b2 (times C, as forces F = -dU/dx for
// U = -C (...), and the moment gradients of -C sf c.E), all vectors in cell
// order (a2, b2 may be null): the TCG-1 and two-field gradients through the
// kernels above in their bilinear mode. Reciprocal part: the gradients of c.E
// (weight sf, no quadratic term) and the Hessian contractions
// -(a.H_b + b.H_a) of the pairs. intra_mu (may be null): the two-field
// form's intramolecular term 1/2 d(intra_mu . (E_s - E_0)) (scale intra_s).
int bilinear_forces(amp_ctx* c, const double4_32a* cv, double sf, const double4_32a* a1, const double4_32a* b1,
                    const double4_32a* a2, const double4_32a* b2, double* F, double* gq, double* gd, double* gt,
                    const double4_32a* intra_mu, double intra_s) {
  const bool fp32 = c->cfg.precision == AMP_MIXED;
  int r;
  pme_theta64(c, c->stream);
  if ((r = force_buffers(c))) return r;
  const long long ng = (long long)c->K * c->K * c->K;
  if (fp32 && !c->grid32b && (r = dev_alloc(c, &c->grid32b, ng))) return r;
  FGeom g;
  const double b = c->cfg.ewald_beta;
  g.L = c->cfg.box;
  g.beta = b;
  g.twob2 = 2.0 * b * b;
  g.gpre = 2.0 * b * b / (b * kSqrtPi);
  g.selfc = 4.0 * b * b * b / (3.0 * kSqrtPi);
  cudaStream_t st = c->stream;
  const dim3 rgrid(amp_blocks((long long)c->n * kGroup, 128));
  const double4_32a* xs[4] = {b1, a1, b2, a2};  // grid of x, contracted with y
  const double4_32a* ys[4] = {a1, b1, a2, b2};
  PhaseScope ps(c, AMP_PHASE_FORCES);
  if (fp32) {
    launch_to32(c, cv, c->p32);
    if ((r = pme_potential(c, true, false, cv, c->p32, c->grid32, st))) return r;
    if ((r = pme_potential(c, true, true, nullptr, nullptr, c->grid32b, st))) return r;
    c->n_launch += 1;
    k_recip_gradients<float><<<rgrid, 128, 0, st>>>(c->n, c->theta32, c->gbase, c->grid32, c->grid32b, c->K, cv,
                                                    c->atomA, c->atomB, c->atomC, c->atomD, sf, 0.0, c->force_recip);
    for (int k = 0; k < 4; ++k) {
      if (!xs[k]) continue;
      launch_to32(c, xs[k], c->p32);
      if ((r = pme_potential(c, true, false, xs[k], c->p32, c->grid32, st))) return r;
      c->n_launch += 1;
      k_recip_hessian_dot<float><<<rgrid, 128, 0, st>>>(c->n, c->theta32, c->gbase, c->grid32, c->K, ys[k],
                                                        c->force_recip);
    }
  } else {
    if ((r = pme_potential(c, false, false, cv, nullptr, c->grid64, st))) return r;
    if ((r = pme_potential(c, false, true, nullptr, nullptr, c->grid64b, st))) return r;
    c->n_launch += 1;
    k_recip_gradients<double><<<rgrid, 128, 0, st>>>(c->n, c->theta, c->gbase, c->grid64, c->grid64b, c->K, cv,
                                                     c->atomA, c->atomB, c->atomC, c->atomD, sf, 0.0,
                                                     c->force_recip);
    for (int k = 0; k < 4; ++k) {
      if (!xs[k]) continue;
      if ((r = pme_potential(c, false, false, xs[k], nullptr, c->grid64, st))) return r;
      c->n_launch += 1;
      k_recip_hessian_dot<double><<<rgrid, 128, 0, st>>>(c->n, c->theta, c->gbase, c->grid64, c->K, ys[k],
                                                         c->force_recip);
    }
  }
  if (c->n_half > 0) {
    c->n_launch += 1;
    const Bilinear bl{a1, b1, a2, b2, sf};
    if (fp32)
      k_pair_forces<float, true><<<amp_blocks(c->n_half, 256), 256, 0, st>>>(
          c->n_half, c->half_i, c->half_j, c->atomA, c->atomB, c->atomC, c->atomD, cv, g, bl, c->force_pair);
    else
      k_pair_forces<double, true><<<amp_blocks(c->n_half, 256), 256, 0, st>>>(
          c->n_half, c->half_i, c->half_j, c->atomA, c->atomB, c->atomC, c->atomD, cv, g, bl, c->force_pair);
    if (intra_mu) {
      c->n_launch += 1;
      k_intra_pair_grads<<<4 * c->n_sm, 128, 0, st>>>(c->intra, c->half_i, c->half_j, c->atomA, c->atomB, c->atomC,
                                                      c->atomD, intra_mu, g, intra_s, c->force_pair);
    }
  }
  c->n_launch += 1;
  k_force_rows<<<amp_blocks((long long)c->n * kRowGroup, 256), 256, 0, st>>>(
      c->n, c->full_start, c->full_ref, c->force_pair, c->force_recip, cv, g.selfc * sf, c->perm, F, gq, gd, gt);
  return cuda_check(c, cudaGetLastError(), "bilinear forces launch");
}

// Gradients of the two-field energy U = -1/2 C mu_d . E_p at the two
// solutions (A mu_d = E_d, A mu_p = E_p; E_p with scale s for two sites of
// one molecule):
//   F = 1/2 C [ d((mu_p + mu_d) . E_d) + d(mu_d . (E_p - E_d)) + d(mu_p . T mu_d) ],
//   dU/dM = -1/2 C d((mu_p + mu_d) . E_d + mu_d . (E_p - E_d))/dM.
int two_rhs_forces(amp_ctx* c, double s, const double4_32a* mu_d, const double4_32a* mu_p, double4_32a* work,
                   double* F, double* gq, double* gd, double* gt) {
  double4_32a* csum = work;        // mu_p + mu_d
  double4_32a* half_p = work + c->n;  // mu_p / 2
  c->n_launch += 1;
  k_two_rhs_vectors<<<amp_blocks(c->n, 256), 256, 0, c->stream>>>(c->n, mu_d, mu_p, csum, half_p);
  return bilinear_forces(c, csum, 0.5, half_p, mu_d, nullptr, nullptr, F, gq, gd, gt, mu_d, s);
}

}  // namespace amp
