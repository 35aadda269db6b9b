// Permanent-multipole energy and its gradients: the interaction of the
// permanent multipoles with each other, the paper's "empole1" (Section
// "Hotspots": the second electrostatic routine of an AMOEBA step beside the
// polarization ones). Charges, dipoles and traceless quadrupoles in the global
// frame, so there are no torques. Everything here runs in float64.
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

struct MGeom {
  double L, beta, twob2, gpre;
};

__device__ __forceinline__ double min_image(double d, double L) { return d - L * rint(d / L); }

// Theta (xx, yy, zz, xy, xz, yz) times v
__device__ __forceinline__ void th_mul(const double* t, const double* v, double* o) {
  o[0] = t[0] * v[0] + t[3] * v[1] + t[4] * v[2];
  o[1] = t[3] * v[0] + t[1] * v[1] + t[5] * v[2];
  o[2] = t[4] * v[0] + t[5] * v[1] + t[2] * v[2];
}

__device__ __forceinline__ double dot3(const double* a, const double* b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// Derivatives of the pair energy in the moments of the field-point site, for
// a source (q, d, Theta) at displacement r (field point minus source):
//   o[0]    = q b0 + (d.r) b1 + (r.Th.r) b2/3
//   o[1..3] = -q b1 r + b1 d - (d.r) b2 r + 2/3 b2 Th r - (r.Th.r) b3 r/3
//   o[4..9] = E_ab for ab = xx, yy, zz, xy, xz, yz (off-diagonals doubled),
//     E_ab = b2 [q r_a r_b/3 - (d_a r_b + d_b r_a)/3 + 2/9 Th_ab]
//          + b3 [(d.r) r_a r_b/3 - 2/9 (r_a (Th r)_b + (Th r)_a r_b)] + b4 (r.Th.r) r_a r_b/9
__device__ __forceinline__ void moment_jet(const double* r, double q, const double* d, const double* th,
                                           const double* b, double* o) {
  double t[3];
  th_mul(th, r, t);
  const double dr = dot3(d, r), trr = dot3(t, r);
  o[0] = q * b[0] + dr * b[1] + trr * b[2] * (1.0 / 3.0);
  const double rad = -q * b[1] - dr * b[2] - trr * b[3] * (1.0 / 3.0);
  for (int a = 0; a < 3; ++a) o[1 + a] = rad * r[a] + b[1] * d[a] + (2.0 / 3.0) * b[2] * t[a];
  const int ia[6] = {0, 1, 2, 0, 0, 1}, ib[6] = {0, 1, 2, 1, 2, 2};
  const double c0 = b[2] * q * (1.0 / 3.0) + b[3] * dr * (1.0 / 3.0) + b[4] * trr * (1.0 / 9.0);
  for (int k = 0; k < 6; ++k) {
    const int a = ia[k], bb = ib[k];
    const double e = c0 * r[a] * r[bb] - b[2] * (1.0 / 3.0) * (d[a] * r[bb] + d[bb] * r[a]) +
                     b[2] * (2.0 / 9.0) * th[k] - b[3] * (2.0 / 9.0) * (r[a] * t[bb] + t[a] * r[bb]);
    o[4 + k] = k < 3 ? e : 2.0 * e;
  }
}

// One thread per unique pair: the force on i (F_j = -F_i) and the moment
// derivatives of both ends, in the backward per-pair record
// [force(3), unused, i's derivatives(10), j's derivatives(10)], units of C.
__global__ void __launch_bounds__(256) k_mpole_pairs(long long nh, const int* __restrict__ half_i,
                                                     const int* __restrict__ half_j,
                                                     const double4_32a* __restrict__ A,
                                                     const double4_32a* __restrict__ B,
                                                     const double4_32a* __restrict__ C,
                                                     const double4_32a* __restrict__ D, MGeom g,
                                                     double* __restrict__ out) {
  const long long pid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (pid >= nh) return;
  const int i = half_i[pid], j = half_j[pid];
  const double4_32a ai = A[i], aj = A[j], bi = B[i], bj = B[j], ci = C[i], cj = C[j], di = D[i], dj = D[j];
  const double r[3] = {min_image(ai.x - aj.x, g.L), min_image(ai.y - aj.y, g.L), min_image(ai.z - aj.z, g.L)};
  const double nr[3] = {-r[0], -r[1], -r[2]};
  const double r2 = dot3(r, r), rr = sqrt(r2), ir = 1.0 / rr, ir2 = ir * ir;
  const double br = g.beta * rr;
  double b[6];
  double fac = exp(-br * br) * g.gpre;
  b[0] = erfc(br) * ir;
  for (int n = 1; n < 6; ++n) {
    b[n] = ((2 * n - 1) * b[n - 1] + fac) * ir2;
    fac *= g.twob2;
  }
  if (di.w == dj.w) {  // same molecule: remove the bare kernels
    double e = ir;
    b[0] -= e;
    for (int n = 1; n < 6; ++n) {
      e *= (2 * n - 1) * ir2;
      b[n] -= e;
    }
  }
  const double qi = ai.w, qj = aj.w;
  const double dpi[3] = {bi.x, bi.y, bi.z}, dpj[3] = {bj.x, bj.y, bj.z};
  const double thi[6] = {ci.x, ci.y, ci.z, ci.w, di.x, di.y};
  const double thj[6] = {cj.x, cj.y, cj.z, cj.w, dj.x, dj.y};
  double ti[3], tj[3];
  th_mul(thi, r, ti);
  th_mul(thj, r, tj);
  const double dir = dot3(dpi, r), djr = dot3(dpj, r), tir = dot3(ti, r), tjr = dot3(tj, r);
  const double thth = thi[0] * thj[0] + thi[1] * thj[1] + thi[2] * thj[2] +
                      2.0 * (thi[3] * thj[3] + thi[4] * thj[4] + thi[5] * thj[5]);
  const double G0 = qi * qj;
  const double G1 = qi * djr - qj * dir + dot3(dpi, dpj);
  const double G2 = -dir * djr + (qi * tjr + qj * tir) * (1.0 / 3.0) + (2.0 / 3.0) * (dot3(dpi, tj) - dot3(dpj, ti)) +
                    (2.0 / 9.0) * thth;
  const double G3 = (djr * tir - dir * tjr) * (1.0 / 3.0) - (4.0 / 9.0) * dot3(ti, tj);
  const double G4 = tir * tjr * (1.0 / 9.0);
  const double rad = G0 * b[1] + G1 * b[2] + G2 * b[3] + G3 * b[4] + G4 * b[5];
  double tjdi[3], tidj[3], titj[3], tjti[3];
  th_mul(thj, dpi, tjdi);
  th_mul(thi, dpj, tidj);
  th_mul(thi, tj, titj);
  th_mul(thj, ti, tjti);
  double* o = out + (long long)kForcePairStride * pid;
  for (int a = 0; a < 3; ++a) {
    const double g1 = qi * dpj[a] - qj * dpi[a];
    const double g2 = -(dpi[a] * djr + dpj[a] * dir) + (2.0 / 3.0) * (qi * tj[a] + qj * ti[a]) +
                      (2.0 / 3.0) * (tjdi[a] - tidj[a]);
    const double g3 = -(2.0 * tj[a] * dir + tjr * dpi[a]) * (1.0 / 3.0) + (dpj[a] * tir + 2.0 * djr * ti[a]) * (1.0 / 3.0) -
                      (4.0 / 9.0) * (titj[a] + tjti[a]);
    const double g4 = (2.0 / 9.0) * (ti[a] * tjr + tj[a] * tir);
    o[a] = rad * r[a] - (b[1] * g1 + b[2] * g2 + b[3] * g3 + b[4] * g4);
  }
  o[3] = 0.0;
  moment_jet(r, qj, dpj, thj, b, o + 4);    // at i, of j
  moment_jet(nr, qi, dpi, thi, b, o + 14);  // at j, of i
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

__device__ __forceinline__ double gsum(double v) {
  const unsigned mask = ((1u << kRowGroup) - 1u) << ((threadIdx.x & 31) & ~(kRowGroup - 1));
#pragma unroll
  for (int o = kRowGroup / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o, kRowGroup);
  return v;
}

struct SelfTerms {
  double q, d, th, bg;  // dU/dq = q*q_i + bg*Q_tot, dU/dd = d*d_i, dU/dTheta_ab = th*Theta_ab
};

// Row sums of the per-pair records + reciprocal + self + background, times C,
// quadrupole diagonal projected; outputs in caller order; per-atom energy
// 1/2 (q dU/dq + d.dU/dd + Theta.dU/dTheta) in sorted order.
__global__ void __launch_bounds__(256) k_mpole_rows(int n, const int* __restrict__ full_start,
                                                    const int* __restrict__ full_ref, const double* __restrict__ pair,
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
  double acc[13];
  for (int k = 0; k < 13; ++k) acc[k] = 0.0;
  const int e = full_start[i + 1];
  for (int k = full_start[i] + l; k < e; k += kRowGroup) {
    const int ref = full_ref[k];
    const double* p = pair + (long long)kForcePairStride * (ref >> 1);
    const double sgn = (ref & 1) ? -1.0 : 1.0;
    acc[0] += sgn * p[0];
    acc[1] += sgn * p[1];
    acc[2] += sgn * p[2];
    const double* g = p + 4 + 10 * (ref & 1);
    for (int m = 0; m < 10; ++m) acc[3 + m] += g[m];
  }
  for (int k = 0; k < 13; ++k) acc[k] = gsum(acc[k]);
  if (l != 0) return;
  const double* rc = recip + (long long)kForceAtomStride * i;
  for (int k = 0; k < 13; ++k) acc[k] += rc[k];
  const double4_32a a = A[i], b = B[i], c = C[i], d = D[i];
  const double th[6] = {c.x, c.y, c.z, c.w, d.x, d.y};
  acc[3] += st.q * a.w + st.bg * (*qtot);
  acc[4] += st.d * b.x;
  acc[5] += st.d * b.y;
  acc[6] += st.d * b.z;
  for (int k = 0; k < 6; ++k) acc[7 + k] += (k < 3 ? 1.0 : 2.0) * st.th * th[k];
  for (int k = 0; k < 13; ++k) acc[k] *= kCoulomb;
  const double mean = (acc[7] + acc[8] + acc[9]) * (1.0 / 3.0);
  acc[7] -= mean;
  acc[8] -= mean;
  acc[9] -= mean;
  double u = a.w * acc[3] + b.x * acc[4] + b.y * acc[5] + b.z * acc[6];
  for (int k = 0; k < 6; ++k) u += th[k] * acc[7 + k];
  e_atom[i] = 0.5 * u;
  const int o = perm[i];
  if (F) {
    F[3 * o] = acc[0];
    F[3 * o + 1] = acc[1];
    F[3 * o + 2] = acc[2];
  }
  if (gq) gq[o] = acc[3];
  if (gd) {
    gd[3 * o] = acc[4];
    gd[3 * o + 1] = acc[5];
    gd[3 * o + 2] = acc[6];
  }
  if (gt)
    for (int k = 0; k < 6; ++k) gt[6 * o + k] = acc[7 + k];
}

}  // namespace

int multipole_energy(amp_ctx* c, double* U, double* F, double* gq, double* gd, double* gt) {
  int r;
  pme_theta64(c);
  if ((r = force_buffers(c))) return r;
  if (c->mpole_e_cap < c->n_cap) {
    dev_free(c, c->mpole_e);
    c->mpole_e = nullptr;
    if ((r = dev_alloc(c, &c->mpole_e, c->n_cap))) return r;
    c->mpole_e_cap = c->n_cap;
  }
  const double b = c->cfg.ewald_beta, L = c->cfg.box;
  MGeom g;
  g.L = L;
  g.beta = b;
  g.twob2 = 2.0 * b * b;
  g.gpre = 2.0 * b / kSqrtPi;
  const double c0 = 2.0 * b / kSqrtPi;
  SelfTerms st;
  st.q = -c0;
  st.d = -c0 * (2.0 * b * b / 3.0);
  st.th = -c0 * (8.0 * b * b * b * b / 45.0);
  st.bg = -3.14159265358979323846 / (L * L * L * b * b);
  cudaStream_t s = c->stream;
  {
    PhaseScope ps(c, AMP_PHASE_FORCES);
    if ((r = pme_potential(c, false, true, nullptr, nullptr, c->grid64b))) return r;
    c->n_launch += 2;
    k_recip_mpole<<<amp_blocks((long long)c->n * kGroup, 128), 128, 0, s>>>(
        c->n, c->theta, c->gbase, c->grid64b, c->K, c->atomA, c->atomB, c->atomC, c->atomD, c->force_recip);
    k_block_sum<<<1, 1024, 0, s>>>(c->n, reinterpret_cast<const double*>(c->atomA) + 3, 4, c->scal + 4);
    if (c->n_half > 0) {
      c->n_launch += 1;
      k_mpole_pairs<<<amp_blocks(c->n_half, 256), 256, 0, s>>>(c->n_half, c->half_i, c->half_j, c->atomA, c->atomB,
                                                               c->atomC, c->atomD, g, c->force_pair);
    }
    c->n_launch += 2;
    k_mpole_rows<<<amp_blocks((long long)c->n * kRowGroup, 256), 256, 0, s>>>(
        c->n, c->full_start, c->full_ref, c->force_pair, c->force_recip, c->atomA, c->atomB, c->atomC, c->atomD,
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
