// Real-space pair terms (kernels b' and b).
//
// The right-hand side of the polarization equation (paper, Section "Hotspots":
// efld0_direct2) and the real-space part of the matrix-vector product applied
// at every solver iteration (tmatxb_pme2) are sums over neighbour pairs. The
// paper's CPU code recomputes every pair quantity on the fly at each call
// (Section "General Structure"). Here every quantity that depends only on the
// geometry is computed once per geometry, for each unique pair:
//   - the damped dipole-field tensor T_ij = -B1u I + B2u r r^T (6 numbers),
//     B1u = B1 - (1 - l3) / r^3, B2u = B2 - 3 (1 - l5) / r^5;
//   - the permanent field of j at i and of i at j, with the intramolecular
//     exclusion (s = 0: B_n - bare_n) and Thole damping (s = 1).
// B_0 = erfc(beta r)/r, B_n = [(2n-1) B_{n-1} + (2 beta^2)^n e^{-beta^2 r^2}/(beta sqrt(pi))]/r^2;
// Thole x = a r^3 / sqrt(alpha_i alpha_j), a = min(a_i, a_j):
// 1 - l3 = e^-x, 1 - l5 = (1 + x) e^-x, 1 - l7 = (1 + x + 0.6 x^2) e^-x.
// On GB300 float64 arithmetic is scarce while HBM is plentiful, so storing
// 6 + 6 numbers per pair and streaming them at every iteration replaces the
// erfc/exp work of the paper's per-call recomputation.
//
// Each iteration then reduces over the full neighbour rows: a group of
// kRowGroup lanes per atom sums T_ij v_j, no atomics, fixed order.
#include <algorithm>
#include <cmath>
#include <vector>

#include "amp_internal.cuh"

namespace amp {
namespace {

struct PairGeom {
  double L, invL, beta, twob2, gpre, selfc;
};

template <typename R>
struct Kern {
  R b1e, b2e, b3e;  // permanent-field coefficients (exclusion applied)
  R b1u, b2u;       // dipole-field coefficients
};

// Field at displacement r (field point minus source) of a multipole:
// E = q B1 r - B1 d + B2 (d.r) r - 2/3 B2 Theta r + 1/3 B3 (r.Theta.r) r
template <typename R>
__device__ __forceinline__ void multipole_field(R rx, R ry, R rz, R q, R dx, R dy, R dz, R qxx, R qyy, R qzz,
                                                R qxy, R qxz, R qyz, R b1, R b2, R b3, R& ex, R& ey, R& ez) {
  const R tx = qxx * rx + qxy * ry + qxz * rz;
  const R ty = qxy * rx + qyy * ry + qyz * rz;
  const R tz = qxz * rx + qyz * ry + qzz * rz;
  const R rtr = rx * tx + ry * ty + rz * tz;
  const R dr = dx * rx + dy * ry + dz * rz;
  const R rad = q * b1 + b2 * dr + b3 * rtr * (R)(1.0 / 3.0);
  const R c2 = b2 * (R)(2.0 / 3.0);
  ex = rad * rx - b1 * dx - c2 * tx;
  ey = rad * ry - b1 * dy - c2 * ty;
  ez = rad * rz - b1 * dz - c2 * tz;
}

// ---- mixed path: pair terms in float32

struct PairGeom32 {
  float beta, twob2, gpre;
};

// Kernel coefficients of one pair in float32.
__device__ __forceinline__ Kern<float> pair_kernels32(float r2, float ai_isa, float aj_isa, float thi, float thj,
                                                      bool same_mol, const PairGeom32& g) {
  Kern<float> k;
  const float r = sqrtf(r2);
  const float ir = 1.f / r;
  const float ir2 = ir * ir;
  const float br = g.beta * r;
  const float ex2 = expf(-br * br);
  const float b0 = erfcf(br) * ir;
  float fac = ex2 * g.gpre;  // e^{-b^2 r^2} / (beta sqrt(pi)) * (2 beta^2)
  const float b1 = (b0 + fac) * ir2;
  fac *= g.twob2;
  const float b2 = (3.f * b1 + fac) * ir2;
  fac *= g.twob2;
  const float b3 = (5.f * b2 + fac) * ir2;
  const float bare1 = ir * ir2;
  const float bare2 = 3.f * bare1 * ir2;
  const float bare3 = 5.f * bare2 * ir2;
  const float x = fminf(thi, thj) * r2 * r * ai_isa * aj_isa;
  const float e = expf(-x);
  const float d3 = e, d5 = (1.f + x) * e, d7 = (1.f + x + 0.6f * x * x) * e;
  k.b1u = b1 - d3 * bare1;
  k.b2u = b2 - d5 * bare2;
  if (same_mol) {
    k.b1e = b1 - bare1;
    k.b2e = b2 - bare2;
    k.b3e = b3 - bare3;
  } else {
    k.b1e = b1 - d3 * bare1;
    k.b2e = b2 - d5 * bare2;
    k.b3e = b3 - d7 * bare3;
  }
  return k;
}

// ---- float64 path of the pair build, entirely in double-float on the float
// units: the minimum image from split positions, 1/r by Newton steps,
// exp(-beta^2 r^2) and the Thole exponential by table-driven reduction, and
// erfc(beta r) = erfcx(beta r) exp(-beta^2 r^2) with erfcx from a per-interval
// Taylor table (df_rsqrt, df_exp_neg, df_erfcx). Per-atom inputs come
// pre-split (pd: position, 1/sqrt(alpha), Thole a, molecule; mp_df: q, d,
// Theta); outputs stay split: the tensor as read by k_t_real_df, the fields
// as Ep[pid] = 12 floats (side 0 x,y,z hi/lo, then side 1).
struct PairGeomDf {
  dflt L, beta, twob2, gpre;
  float invL;
};

// minimum-image component: the pair lies within rc < L/2, so rounding d/L
// from the hi part picks the same image as exact arithmetic would
__device__ __forceinline__ dflt min_image_df(dflt d, const PairGeomDf& g) {
  const float sh = rintf(d.hi * g.invL);
  return sh == 0.f ? d : df_sub(d, df_mul({sh, 0.f}, g.L));
}

// A pair of two sites of one molecule joins the list intra ([0] count, then
// pair ids; one atomic per warp): the float64 permanent-field terms
// (k_intra_fields64) and the scaled fields of the two-field form use it.
__device__ __forceinline__ void append_intra(bool same, long long pid, int* __restrict__ intra) {
  const unsigned live = __activemask();
  const unsigned m = __ballot_sync(live, same);
  if (m) {
    const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(intra, __popc(m));
    base = __shfl_sync(live, base, leader);
    if (same) intra[1 + base + __popc(m & ((1u << lane) - 1u))] = (int)pid;
  }
}

// Mixed path pair build: the displacement from the split positions (minimum
// image in double-float, then rounded to float), every other quantity in
// float32 from the float parts of the per-atom records (pd, mp_df), so that
// no float64 instruction is issued. Writes the tensor to both full-list
// entries of the pair (the owner's and the transposed one, as the float64
// path does), so that the product kernel reads each row's tensors
// contiguously, and both permanent fields, in float32.
__global__ void __launch_bounds__(256) k_pair_build32(long long nh, const int* __restrict__ half_i,
                                                      const int* __restrict__ half_j, const float4* __restrict__ pd,
                                                      const float4* __restrict__ mp_df, PairGeomDf gd, PairGeom32 g,
                                                      const int* __restrict__ full_start,
                                                      const int* __restrict__ half_start,
                                                      const int* __restrict__ pos_tr, float4* __restrict__ T4,
                                                      float2* __restrict__ T2, float* __restrict__ Ep,
                                                      int* __restrict__ intra) {
  const long long pid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (pid >= nh) return;
  const int i = half_i[pid], j = half_j[pid];
  const float4 hi_i = pd[3 * (long long)i], lo_i = pd[3 * (long long)i + 1], th_i = pd[3 * (long long)i + 2];
  const float4 hi_j = pd[3 * (long long)j], lo_j = pd[3 * (long long)j + 1], th_j = pd[3 * (long long)j + 2];
  append_intra(__float_as_int(th_i.z) == __float_as_int(th_j.z), pid, intra);
  const dflt dx = min_image_df(df_sub({hi_i.x, lo_i.x}, {hi_j.x, lo_j.x}), gd);
  const dflt dy = min_image_df(df_sub({hi_i.y, lo_i.y}, {hi_j.y, lo_j.y}), gd);
  const dflt dz = min_image_df(df_sub({hi_i.z, lo_i.z}, {hi_j.z, lo_j.z}), gd);
  const float rx = dx.hi + dx.lo, ry = dy.hi + dy.lo, rz = dz.hi + dz.lo;
  const float r2 = rx * rx + ry * ry + rz * rz;
  const Kern<float> k = pair_kernels32(r2, hi_i.w, hi_j.w, th_i.x, th_j.x,
                                       __float_as_int(th_i.z) == __float_as_int(th_j.z), g);
  {
    const float4 ta = make_float4(k.b2u * rx * rx - k.b1u, k.b2u * ry * ry - k.b1u, k.b2u * rz * rz - k.b1u,
                                  k.b2u * rx * ry);
    const float2 tb = make_float2(k.b2u * rx * rz, k.b2u * ry * rz);
    const long long k1 = full_start[i] + (pid - half_start[i]), k2 = pos_tr[pid];
    T4[k1] = ta;
    T2[k1] = tb;
    T4[k2] = ta;
    T2[k2] = tb;
  }
  // float parts of q, d, Theta (mp_df: (q, dx), (dy, dz), (Qxx, Qyy), (Qzz, Qxy), (Qxz, Qyz) as hi/lo)
  const float4* mi = mp_df + 5 * (long long)i;
  const float4* mj = mp_df + 5 * (long long)j;
  const float4 i0 = mi[0], i1 = mi[1], i2 = mi[2], i3 = mi[3], i4 = mi[4];
  const float4 j0 = mj[0], j1 = mj[1], j2 = mj[2], j3 = mj[3], j4 = mj[4];
  float ex, ey, ez;
  multipole_field<float>(rx, ry, rz, j0.x, j0.z, j1.x, j1.z, j2.x, j2.z, j3.x, j3.z, j4.x, j4.z, k.b1e, k.b2e,
                         k.b3e, ex, ey, ez);
  float* e = Ep + 6 * pid;
  e[0] = ex;
  e[1] = ey;
  e[2] = ez;
  multipole_field<float>(-rx, -ry, -rz, i0.x, i0.z, i1.x, i1.z, i2.x, i2.z, i3.x, i3.z, i4.x, i4.z, k.b1e, k.b2e,
                         k.b3e, ex, ey, ez);
  e[3] = ex;
  e[4] = ey;
  e[5] = ez;
}

// The geometry-only terms of pair (i, j) in double-float: r = x_i - x_j
// (minimum image), 1/r, the screened kernels B1..B3, the bare kernels and the
// Thole exponent x with e^-x.
struct PairTermsDf {
  dflt R[3], IR2, B1, B2, B3, bare1, bare2, bare3, X, E;
};

__device__ __forceinline__ PairTermsDf pair_terms_df(const float4& hi_i, const float4& lo_i, const float4& th_i,
                                                     const float4& hi_j, const float4& lo_j, const float4& th_j,
                                                     const PairGeomDf& g, const float2* __restrict__ tab) {
  PairTermsDf p;
  p.R[0] = min_image_df(df_sub({hi_i.x, lo_i.x}, {hi_j.x, lo_j.x}), g);
  p.R[1] = min_image_df(df_sub({hi_i.y, lo_i.y}, {hi_j.y, lo_j.y}), g);
  p.R[2] = min_image_df(df_sub({hi_i.z, lo_i.z}, {hi_j.z, lo_j.z}), g);
  const dflt R2 = df_madd(p.R[2], p.R[2], df_madd(p.R[1], p.R[1], df_mul(p.R[0], p.R[0])));
  const dflt IR = df_rsqrt(R2);
  const dflt RR = df_mul(R2, IR);
  const dflt BR = df_mul(g.beta, RR);
  const dflt E2 = df_exp_neg(df_mul(BR, BR), tab);  // exp(-beta^2 r^2)
  const dflt B0 = df_mul(df_mul(df_erfcx(BR, tab), E2), IR);
  dflt FAC = df_mul(E2, g.gpre);
  // Thole: x = a r^3 / sqrt(alpha_i alpha_j), a = min(a_i, a_j)
  const dflt A = th_i.x < th_j.x || (th_i.x == th_j.x && th_i.y <= th_j.y) ? dflt{th_i.x, th_i.y}
                                                                           : dflt{th_j.x, th_j.y};
  p.X = df_mul(df_mul(A, df_mul(R2, RR)), df_mul({hi_i.w, lo_i.w}, {hi_j.w, lo_j.w}));
  p.E = df_exp_neg(p.X, tab);
  const dflt THREE = {3.f, 0.f}, FIVE = {5.f, 0.f};
  p.IR2 = df_mul(IR, IR);
  p.B1 = df_mul(df_add(B0, FAC), p.IR2);
  FAC = df_mul(FAC, g.twob2);
  p.B2 = df_mul(df_madd(THREE, p.B1, FAC), p.IR2);
  FAC = df_mul(FAC, g.twob2);
  p.B3 = df_mul(df_madd(FIVE, p.B2, FAC), p.IR2);
  p.bare1 = df_mul(IR, p.IR2);
  p.bare2 = df_mul(df_mul(THREE, p.bare1), p.IR2);
  p.bare3 = df_mul(df_mul(FIVE, p.bare2), p.IR2);
  return p;
}

__global__ void __launch_bounds__(256) k_pair_build_df(long long nh, const int* __restrict__ half_i,
                                                       const int* __restrict__ half_j,
                                                       const float4* __restrict__ pd,
                                                       const float4* __restrict__ mp_df, PairGeomDf g,
                                                       const float2* __restrict__ tab,
                                                       const int* __restrict__ full_start,
                                                       const int* __restrict__ half_start,
                                                       const int* __restrict__ pos_tr, float4* __restrict__ C64,
                                                       float* __restrict__ Ep, int* __restrict__ intra) {
  const long long pid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (pid >= nh) return;
  const int i = half_i[pid], j = half_j[pid];
  const float4 hi_i = pd[3 * (long long)i], lo_i = pd[3 * (long long)i + 1], th_i = pd[3 * (long long)i + 2];
  const float4 hi_j = pd[3 * (long long)j], lo_j = pd[3 * (long long)j + 1], th_j = pd[3 * (long long)j + 2];
  append_intra(__float_as_int(th_i.z) == __float_as_int(th_j.z), pid, intra);
  const PairTermsDf p = pair_terms_df(hi_i, lo_i, th_i, hi_j, lo_j, th_j, g, tab);
  const dflt(&R)[3] = p.R;
  const dflt NR[3] = {df_neg(R[0]), df_neg(R[1]), df_neg(R[2])};
  const dflt X = p.X, E = p.E, B1 = p.B1, B2 = p.B2, B3 = p.B3;
  const dflt bare1 = p.bare1, bare2 = p.bare2, bare3 = p.bare3;
  const dflt ONE = {1.f, 0.f};
  const dflt d3 = E;
  const dflt d5 = df_mul(df_add(ONE, X), E);
  const dflt six = {0.600000024f, -2.38418579e-08f};  // 0.6 = hi + lo
  const dflt d7 = df_mul(df_madd(df_mul(six, X), X, df_add(ONE, X)), E);
  const dflt b1u = df_sub(B1, df_mul(d3, bare1));
  const dflt b2u = df_sub(B2, df_mul(d5, bare2));
  dflt b1e, b2e, b3e;
  if (__float_as_int(th_i.z) == __float_as_int(th_j.z)) {  // same molecule
    b1e = df_sub(B1, bare1);
    b2e = df_sub(B2, bare2);
    b3e = df_sub(B3, bare3);
  } else {
    b1e = b1u;
    b2e = b2u;
    b3e = df_sub(B3, df_mul(d7, bare3));
  }
  // the tensor T = -b1u I + b2u r r^T as its two scalars, in both full-list
  // entries of the pair (the owner's and the transposed one), so that the
  // product kernel reads every row's entries contiguously (16 bytes each)
  // and rebuilds r from the positions as above
  {
    const float4 t = make_float4(b1u.hi, b1u.lo, b2u.hi, b2u.lo);
    C64[full_start[i] + (pid - half_start[i])] = t;
    C64[pos_tr[pid]] = t;
  }
  // permanent fields: at i from j (r), at j from i (-r)
  dflt mpi[10], mpj[10];
  {
    const float4* pi = mp_df + 5 * (long long)i;
    const float4* pj = mp_df + 5 * (long long)j;
    for (int k = 0; k < 5; ++k) {
      const float4 u = pi[k], w = pj[k];
      mpi[2 * k] = {u.x, u.y};
      mpi[2 * k + 1] = {u.z, u.w};
      mpj[2 * k] = {w.x, w.y};
      mpj[2 * k + 1] = {w.z, w.w};
    }
  }
  dflt fi[3], fj[3];
  mp_field_df(R, mpj, b1e, b2e, b3e, fi);
  mp_field_df(NR, mpi, b1e, b2e, b3e, fj);
  if (__float_as_int(th_i.z) == __float_as_int(th_j.z))  // same molecule: float64, by k_intra_fields64
    for (int a = 0; a < 3; ++a) fi[a] = fj[a] = dflt{0.f, 0.f};
  float4* e = reinterpret_cast<float4*>(Ep + 12 * pid);
  e[0] = make_float4(fi[0].hi, fi[0].lo, fi[1].hi, fi[1].lo);
  e[1] = make_float4(fi[2].hi, fi[2].lo, fj[0].hi, fj[0].lo);
  e[2] = make_float4(fj[1].hi, fj[1].lo, fj[2].hi, fj[2].lo);
}

// Per sorted atom s: mp_df[s] = q, d, Theta as hi/lo float pairs (5 float4);
// pd[s] = (x, y, z, 1/sqrt(alpha)) hi, the same lo, (Thole a hi, lo, molecule, 0);
// xhl[s] (if given) = (x, y, z, 0) hi, the same lo.
__global__ void k_split_multipoles(int n, const double4_32a* __restrict__ A, const double4_32a* __restrict__ B,
                                   const double4_32a* __restrict__ C, const double4_32a* __restrict__ D,
                                   float4* __restrict__ mp, float4* __restrict__ pd, float4* __restrict__ xhl) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const double4_32a a = A[s], b = B[s], c = C[s], d = D[s];
  const double v[10] = {a.w, b.x, b.y, b.z, c.x, c.y, c.z, c.w, d.x, d.y};
  for (int k = 0; k < 5; ++k) {
    const dflt u = df_split(v[2 * k]), w = df_split(v[2 * k + 1]);
    mp[5 * (long long)s + k] = make_float4(u.hi, u.lo, w.hi, w.lo);
  }
  if (pd) {
    const dflt x = df_split(a.x), y = df_split(a.y), z = df_split(a.z), is = df_split(b.w), th = df_split(d.z);
    pd[3 * (long long)s] = make_float4(x.hi, y.hi, z.hi, is.hi);
    pd[3 * (long long)s + 1] = make_float4(x.lo, y.lo, z.lo, is.lo);
    pd[3 * (long long)s + 2] = make_float4(th.hi, th.lo, __int_as_float((int)d.w), 0.f);
    if (xhl) {
      xhl[2 * (long long)s] = make_float4(x.hi, y.hi, z.hi, 0.f);
      xhl[2 * (long long)s + 1] = make_float4(x.lo, y.lo, z.lo, 0.f);
    }
  }
}

// out_i = sum over row entries of the split per-pair fields + add_i (if
// given) + selfc selfv_i. E0: the permanent fields of the pair build (zero
// for two sites of one molecule), add = their float64 intramolecular terms.
__global__ void __launch_bounds__(256) k_row_sum_fields_df(int n, const int* __restrict__ full_start,
                                                           const int* __restrict__ full_ref,
                                                           const float* __restrict__ Ep, double selfc,
                                                           const double4_32a* __restrict__ selfv,
                                                           const double4_32a* __restrict__ add,
                                                           double4_32a* __restrict__ out) {
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = gid / kRowGroup, l = gid % kRowGroup;
  if (i >= n) return;
  dflt sx = {0.f, 0.f}, sy = {0.f, 0.f}, sz = {0.f, 0.f};
  const int e = full_start[i + 1];
  for (int k = full_start[i] + l; k < e; k += kRowGroup) {
    const int ref = full_ref[k];
    const float2* p = reinterpret_cast<const float2*>(Ep + 12 * (long long)(ref >> 1) + 6 * (ref & 1));
    const float2 x = p[0], y = p[1], z = p[2];
    sx = df_add(sx, {x.x, x.y});
    sy = df_add(sy, {y.x, y.y});
    sz = df_add(sz, {z.x, z.y});
  }
  sx = df_group_sum(sx);
  sy = df_group_sum(sy);
  sz = df_group_sum(sz);
  if (l == 0) {
    const double4_32a s = selfv[i];
    const double4_32a a = add ? add[i] : make_double4_32a(0.0, 0.0, 0.0, 0.0);
    out[i] = make_double4_32a(df_to_double(sx) + a.x + selfc * s.x, df_to_double(sy) + a.y + selfc * s.y,
                              df_to_double(sz) + a.z + selfc * s.z, 0.0);
  }
}

__device__ __forceinline__ double group_sum(double v) {
  const unsigned mask = ((1u << kRowGroup) - 1u) << ((threadIdx.x & 31) & ~(kRowGroup - 1));
#pragma unroll
  for (int o = kRowGroup / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o, kRowGroup);
  return v;
}

// Permanent field of the intramolecular pairs (scale 0: the screened kernels
// minus the bare ones, no Thole damping) in float64, one pair per thread over
// the list that the pair build appended (a float64 instruction holds the
// float64 pipe as long for one active lane as for 32, so these pairs are not
// evaluated inside the rows, where they are two in ~70). r = x_i - x_j
// minimum image, B_n by the recurrence above; the fields at i (from j) and
// at j (from i) are added to the per-atom sums out (float64 atomics; a site
// with two partners, as in water, gets the same sum in either order).
__global__ void __launch_bounds__(128) k_intra_fields64(const int* __restrict__ intra,
                                                        const int* __restrict__ half_i,
                                                        const int* __restrict__ half_j, PairGeom g,
                                                        const double4_32a* __restrict__ A,
                                                        const double4_32a* __restrict__ B,
                                                        const double4_32a* __restrict__ C,
                                                        const double4_32a* __restrict__ D,
                                                        double4_32a* __restrict__ out) {
  const int cnt = intra[0];
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < cnt; k += gridDim.x * blockDim.x) {
    const int pid = intra[1 + k];
    const int i = half_i[pid], j = half_j[pid];
    const double4_32a ai = A[i], aj = A[j];
    double r3[3] = {ai.x - aj.x, ai.y - aj.y, ai.z - aj.z};
    for (int a = 0; a < 3; ++a) r3[a] -= g.L * rint(r3[a] * g.invL);
    const double r2 = r3[0] * r3[0] + r3[1] * r3[1] + r3[2] * r3[2];
    const double r = sqrt(r2), ir = 1.0 / r, ir2 = ir * ir;
    const double br = g.beta * r;
    double fac = exp(-br * br) * g.gpre;
    const double b0 = erfc(br) * ir;
    const double B1 = (b0 + fac) * ir2;
    fac *= g.twob2;
    const double B2 = (3.0 * B1 + fac) * ir2;
    fac *= g.twob2;
    const double B3 = (5.0 * B2 + fac) * ir2;
    const double bare1 = ir * ir2, bare2 = 3.0 * bare1 * ir2, bare3 = 5.0 * bare2 * ir2;
    const double b1 = B1 - bare1, b2 = B2 - bare2, b3 = B3 - bare3;
    const double4_32a bi = B[i], bj = B[j], ci = C[i], cj = C[j], di = D[i], dj = D[j];
    double f[6];
    multipole_field<double>(r3[0], r3[1], r3[2], aj.w, bj.x, bj.y, bj.z, cj.x, cj.y, cj.z, cj.w, dj.x, dj.y, b1,
                            b2, b3, f[0], f[1], f[2]);
    multipole_field<double>(-r3[0], -r3[1], -r3[2], ai.w, bi.x, bi.y, bi.z, ci.x, ci.y, ci.z, ci.w, di.x, di.y,
                            b1, b2, b3, f[3], f[4], f[5]);
    double* oi = reinterpret_cast<double*>(out + i);
    double* oj = reinterpret_cast<double*>(out + j);
    for (int a = 0; a < 3; ++a) {
      atomicAdd(oi + a, f[a]);
      atomicAdd(oj + a, f[3 + a]);
    }
  }
}

// The difference between the permanent field with scale s for two sites of
// one molecule and with scale 0 (the two-field form's E_p - E_d): for each
// intramolecular pair the Thole-damped bare field times s, kernels
// s l3 bare1, s l5 bare2, s l7 bare3 (the screened parts cancel), in float64,
// added to out at both ends (float64 atomics).
__global__ void __launch_bounds__(128) k_intra_scaled64(const int* __restrict__ intra, const int* __restrict__ half_i,
                                                        const int* __restrict__ half_j, PairGeom g, double s,
                                                        const double4_32a* __restrict__ A,
                                                        const double4_32a* __restrict__ B,
                                                        const double4_32a* __restrict__ C,
                                                        const double4_32a* __restrict__ D,
                                                        double4_32a* __restrict__ out) {
  const int cnt = intra[0];
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < cnt; k += gridDim.x * blockDim.x) {
    const int pid = intra[1 + k];
    const int i = half_i[pid], j = half_j[pid];
    const double4_32a ai = A[i], aj = A[j], bi = B[i], bj = B[j], ci = C[i], cj = C[j], di = D[i], dj = D[j];
    double r3[3] = {ai.x - aj.x, ai.y - aj.y, ai.z - aj.z};
    if (g.L > 0.0)
      for (int a = 0; a < 3; ++a) r3[a] -= g.L * rint(r3[a] * g.invL);
    const double r2 = r3[0] * r3[0] + r3[1] * r3[1] + r3[2] * r3[2];
    const double r = sqrt(r2), ir = 1.0 / r, ir2 = ir * ir;
    const double bare1 = ir * ir2, bare2 = 3.0 * bare1 * ir2, bare3 = 5.0 * bare2 * ir2;
    const double x = fmin(di.z, dj.z) * r2 * r * bi.w * bj.w;
    const double e = exp(-x);
    const double l3 = 1.0 - e, l5 = 1.0 - (1.0 + x) * e, l7 = 1.0 - (1.0 + x + 0.6 * x * x) * e;
    const double b1 = s * l3 * bare1, b2 = s * l5 * bare2, b3 = s * l7 * bare3;
    double f[6];
    multipole_field<double>(r3[0], r3[1], r3[2], aj.w, bj.x, bj.y, bj.z, cj.x, cj.y, cj.z, cj.w, dj.x, dj.y, b1,
                            b2, b3, f[0], f[1], f[2]);
    multipole_field<double>(-r3[0], -r3[1], -r3[2], ai.w, bi.x, bi.y, bi.z, ci.x, ci.y, ci.z, ci.w, di.x, di.y,
                            b1, b2, b3, f[3], f[4], f[5]);
    double* oi = reinterpret_cast<double*>(out + i);
    double* oj = reinterpret_cast<double*>(out + j);
    for (int a = 0; a < 3; ++a) {
      atomicAdd(oi + a, f[a]);
      atomicAdd(oj + a, f[3 + a]);
    }
  }
}

// The mixed path's float64 residual check: T_ij v_j and T_ij v_i of every
// pair with the tensor recomputed on the fly in double-float (the terms of
// pair_terms_df), v given as hi/lo floats; written in the layout of the
// permanent fields (12 floats per pair) for k_row_sum_fields_df.
__global__ void __launch_bounds__(256) k_pair_tv_df(long long nh, const int* __restrict__ half_i,
                                                    const int* __restrict__ half_j, const float4* __restrict__ pd,
                                                    PairGeomDf g, const float2* __restrict__ tab,
                                                    const float4* __restrict__ vh, const float4* __restrict__ vl,
                                                    float* __restrict__ out) {
  const long long pid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (pid >= nh) return;
  const int i = half_i[pid], j = half_j[pid];
  const float4 hi_i = pd[3 * (long long)i], lo_i = pd[3 * (long long)i + 1], th_i = pd[3 * (long long)i + 2];
  const float4 hi_j = pd[3 * (long long)j], lo_j = pd[3 * (long long)j + 1], th_j = pd[3 * (long long)j + 2];
  const PairTermsDf p = pair_terms_df(hi_i, lo_i, th_i, hi_j, lo_j, th_j, g, tab);
  const dflt b1u = df_sub(p.B1, df_mul(p.E, p.bare1));
  const dflt b2u = df_sub(p.B2, df_mul(df_mul(df_add({1.f, 0.f}, p.X), p.E), p.bare2));
  dflt f[2][3];
  for (int side = 0; side < 2; ++side) {  // field at i from v_j, at j from v_i
    const int o = side == 0 ? j : i;
    const float4 h = vh[o], l = vl[o];
    const dflt v[3] = {{h.x, l.x}, {h.y, l.y}, {h.z, l.z}};
    const dflt s = df_mul(b2u, df_madd(p.R[2], v[2], df_madd(p.R[1], v[1], df_mul(p.R[0], v[0]))));
    for (int a = 0; a < 3; ++a) f[side][a] = df_sub(df_mul(s, p.R[a]), df_mul(b1u, v[a]));
  }
  float4* e = reinterpret_cast<float4*>(out + 12 * pid);
  e[0] = make_float4(f[0][0].hi, f[0][0].lo, f[0][1].hi, f[0][1].lo);
  e[1] = make_float4(f[0][2].hi, f[0][2].lo, f[1][0].hi, f[1][0].lo);
  e[2] = make_float4(f[1][1].hi, f[1][1].lo, f[1][2].hi, f[1][2].lo);
}

// out_i = sum over row entries of the stored per-pair vectors (side-selected)
// + selfc * self_i.xyz. Used for E0 (stored permanent fields) and for the
// float64 direct products.
template <typename R>
__global__ void __launch_bounds__(256) k_row_sum_pairvec(int n, const int* __restrict__ full_start,
                                                         const int* __restrict__ full_ref,
                                                         const R* __restrict__ pv, double selfc,
                                                         const double4_32a* __restrict__ selfv,
                                                         double4_32a* __restrict__ out) {
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = gid / kRowGroup, l = gid % kRowGroup;
  if (i >= n) return;  // whole groups exit together (n rows, kRowGroup | 32)
  double sx = 0, sy = 0, sz = 0;
  const int e = full_start[i + 1];
  for (int k = full_start[i] + l; k < e; k += kRowGroup) {
    const int ref = full_ref[k];
    const R* p = pv + 6 * (long long)(ref >> 1) + 3 * (ref & 1);
    sx += (double)p[0];
    sy += (double)p[1];
    sz += (double)p[2];
  }
  sx = group_sum(sx);
  sy = group_sum(sy);
  sz = group_sum(sz);
  if (l == 0) {
    const double4_32a s = selfv[i];
    out[i] = make_double4_32a(sx + selfc * s.x, sy + selfc * s.y, sz + selfc * s.z, 0.0);
  }
}

// Resident blocks per SM of the real-space products (rows grid-strided, so
// one wave). Float64 path: every block its registers allow (5 at 48
// registers; against 4: water-23556 solve 0.869 vs 0.891 ms, water-96000
// unchanged; a cap above the residency leaves a second, partial wave: 6 gave
// 3.32 vs 2.87 ms there). Mixed: 4 of the 8 the registers allow, which keeps
// room for the reciprocal chain's blocks beside it (5 and 6 measured within
// the noise).
constexpr int kTRealBlocksPerSmDf = 5;
constexpr int kTRealBlocksPerSm32 = 4;

// Real-space T*v of the float64 path in double-float, one row per group of
// kRowGroup lanes, rows grid-strided. Each full-list entry holds the pair's
// two tensor scalars (b1, b2: T = -b1 I + b2 r r^T), 16 bytes read in entry
// order; r = x_i - x_j (minimum image) is rebuilt from the hi/lo positions
// with the pair build's own operations, and T v_j = b2 (r . v_j) r - b1 v_j.
// x_j and v_j (32 bytes each, hi/lo) are gathered per entry; they are shared
// by the ~70 rows that list atom j and stay in L1/L2, so DRAM streams only
// the 20 bytes per entry. Lanes 0..2 finish one component each in float64 (a
// float64 instruction holds the float64 pipe as long for one active lane as
// for 32), adding the self term selfc v_i.
__global__ void __launch_bounds__(256, kTRealBlocksPerSmDf) k_t_real_df(int n, const int* __restrict__ full_start,
                                                   const int* __restrict__ full_j, const float4* __restrict__ C64,
                                                   const float4* __restrict__ xhl, PairGeomDf g, double selfc,
                                                   const float4* __restrict__ vhl,
                                                   const double4_32a* __restrict__ v64, double4_32a* __restrict__ out,
                                                   const int* __restrict__ stop) {
  if (stop && *stop) return;  // the solver has stopped: nothing to compute
  const int l = threadIdx.x % kRowGroup;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) / kRowGroup; i < n; i += gridDim.x * (blockDim.x / kRowGroup)) {
    dflt sx = {0.f, 0.f}, sy = {0.f, 0.f}, sz = {0.f, 0.f};
    float4 xih, xil;
    ld8_ro(xhl + 2 * (long long)i, xih, xil);
    const int e = full_start[i + 1];
    int k = full_start[i] + l;
    int jn = k < e ? __ldcs(full_j + k) : 0;
    for (; k < e; k += kRowGroup) {
      const int j = jn;
      if (k + kRowGroup < e) jn = __ldcs(full_j + k + kRowGroup);
      const float4 cb = __ldcs(C64 + k);
      float4 xh, xl, h, w;
      ld8_ro(xhl + 2 * (long long)j, xh, xl);
      ld8_ro(vhl + 2 * (long long)j, h, w);
      const dflt r0 = min_image_df(df_sub({xih.x, xil.x}, {xh.x, xl.x}), g);
      const dflt r1 = min_image_df(df_sub({xih.y, xil.y}, {xh.y, xl.y}), g);
      const dflt r2 = min_image_df(df_sub({xih.z, xil.z}, {xh.z, xl.z}), g);
      dflt rv = df_mul(r0, {h.x, w.x});
      df_fma(rv, r1.hi, r1.lo, h.y, w.y);
      df_fma(rv, r2.hi, r2.lo, h.z, w.z);
      const dflt q = df_mul({cb.z, cb.w}, rv);  // b2 (r . v)
      const float nbh = -cb.x, nbl = -cb.y;     // -b1
      df_fma(sx, q.hi, q.lo, r0.hi, r0.lo);
      df_fma(sx, nbh, nbl, h.x, w.x);
      df_fma(sy, q.hi, q.lo, r1.hi, r1.lo);
      df_fma(sy, nbh, nbl, h.y, w.y);
      df_fma(sz, q.hi, q.lo, r2.hi, r2.lo);
      df_fma(sz, nbh, nbl, h.z, w.z);
    }
    sx = df_group_sum(sx);
    sy = df_group_sum(sy);
    sz = df_group_sum(sz);
    if (l < 4) {
      double* o = reinterpret_cast<double*>(out + i);
      if (l < 3) {
        const dflt sc = l == 0 ? sx : (l == 1 ? sy : sz);
        o[l] = (double)sc.hi + (double)sc.lo + selfc * reinterpret_cast<const double*>(v64 + i)[l];
      } else {
        o[3] = 0.0;
      }
    }
  }
}

// acc += x, error-free: the rounding error of the float sum goes to acc.lo
// (cascaded summation; acc.hi + acc.lo carries the sum to ~float64 level)
__device__ __forceinline__ void acc_add(dflt& acc, float x) {
  const dflt s = df_two_sum(acc.hi, x);
  acc.hi = s.hi;
  acc.lo = __fadd_rn(acc.lo, s.lo);
}

// Mixed precision: float32 tensors (stored per full-list entry, in row order:
// one 16-byte and one 8-byte load per entry, contiguous across the lanes of a
// row) and the float32 copy of v (a 16-byte gather per entry); each entry's
// field T_ij v_j in float32, summed over the lane's entries with error-free
// two-sums (acc_add), the row total in double-float across the lanes, then
// lanes 0..2 finish one component each in float64 (a float64 instruction
// holds the float64 pipe as long for one active lane as for 32). Rows are
// grid-strided.
__global__ void __launch_bounds__(256) k_t_real32(int n, const int* __restrict__ full_start,
                                                  const int* __restrict__ full_j, const float4* __restrict__ T4,
                                                  const float2* __restrict__ T2, double selfc,
                                                  const float4* __restrict__ v32, const double4_32a* __restrict__ v64,
                                                  double4_32a* __restrict__ out, const int* __restrict__ stop) {
  if (stop && *stop) return;
  const int l = threadIdx.x % kRowGroup;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) / kRowGroup; i < n; i += gridDim.x * (blockDim.x / kRowGroup)) {
    dflt sx = {0.f, 0.f}, sy = {0.f, 0.f}, sz = {0.f, 0.f};
    const int e = full_start[i + 1];
    int k = full_start[i] + l;
    int jn = k < e ? __ldcs(full_j + k) : 0;
    for (; k < e; k += kRowGroup) {
      const int j = jn;
      if (k + kRowGroup < e) jn = __ldcs(full_j + k + kRowGroup);
      const float4 a = __ldcs(T4 + k);  // xx yy zz xy
      const float2 b = __ldcs(T2 + k);  // xz yz
      const float4 vj = v32[j];
      acc_add(sx, fmaf(b.x, vj.z, fmaf(a.w, vj.y, a.x * vj.x)));
      acc_add(sy, fmaf(b.y, vj.z, fmaf(a.y, vj.y, a.w * vj.x)));
      acc_add(sz, fmaf(a.z, vj.z, fmaf(b.y, vj.y, b.x * vj.x)));
    }
    sx = df_group_sum(sx);
    sy = df_group_sum(sy);
    sz = df_group_sum(sz);
    if (l < 4) {
      double* o = reinterpret_cast<double*>(out + i);
      if (l < 3) {
        const dflt d = l == 0 ? sx : (l == 1 ? sy : sz);
        o[l] = df_to_double(d) + selfc * reinterpret_cast<const double*>(v64 + i)[l];
      } else {
        o[3] = 0.0;
      }
    }
  }
}

PairGeom geom(const amp_ctx* c) {
  PairGeom g;
  const double b = c->cfg.ewald_beta;
  g.L = c->cfg.box;
  g.invL = c->cfg.box > 0.0 ? 1.0 / c->cfg.box : 0.0;
  g.beta = b;
  g.twob2 = 2.0 * b * b;
  g.gpre = 2.0 * b * b / (b * kSqrtPi);
  g.selfc = 4.0 * b * b * b / (3.0 * kSqrtPi);
  return g;
}

dflt dsplit_host(double v) {
  const float h = (float)v;
  return {h, (float)(v - (double)h)};
}

PairGeomDf geom_df(const PairGeom& g) {
  PairGeomDf gd;
  gd.L = dsplit_host(g.L);
  gd.beta = dsplit_host(g.beta);
  gd.twob2 = dsplit_host(g.twob2);
  gd.gpre = dsplit_host(g.gpre);
  gd.invL = (float)g.invL;
  return gd;
}

}  // namespace

// Table for df_erfcx and df_exp_neg, built in long double on the host.
// erfcx(x0 + t) = sum_n a_n t^n at the centre x0 of each interval, from the
// differential equation y' = 2 x y - 2/sqrt(pi) of erfcx:
//   a_0 = erfc(x0) exp(x0^2), a_1 = 2 x0 a_0 - 2/sqrt(pi),
//   (n + 1) a_{n+1} = 2 x0 a_n + 2 a_{n-1}  (n >= 1);
// with |t| <= 1/16 the series is cut after t^11 (remainder below 1e-17).
void dfm_host_table(std::vector<float2>& tab) {
  tab.assign(kDfmTableSize, make_float2(0.f, 0.f));
  auto put = [&](int k, long double v) {
    const float h = (float)v;
    tab[k] = make_float2(h, (float)(v - (long double)h));
  };
  const long double two_rsqrtpi = 2.0L / std::sqrt(std::acos(-1.0L));
  for (int i = 0; i < kErfcxIntervals; ++i) {
    const long double x0 = ((long double)i + 0.5L) / 8.0L;
    long double a[kErfcxTerms];
    a[0] = std::erfc(x0) * std::exp(x0 * x0);
    a[1] = 2.0L * x0 * a[0] - two_rsqrtpi;
    for (int n = 1; n + 1 < kErfcxTerms; ++n) a[n + 1] = (2.0L * x0 * a[n] + 2.0L * a[n - 1]) / (long double)(n + 1);
    for (int n = 0; n < kErfcxTerms; ++n) put(i * kErfcxTerms + n, a[n]);
  }
  for (int j = -11; j <= 11; ++j) put(kExpTable + 11 + j, std::exp((long double)j / 32.0L));
}

int dfm_setup(amp_ctx* c) {
  std::vector<float2> tab;
  dfm_host_table(tab);
  int r;
  if (!c->dfm && (r = dev_alloc(c, &c->dfm, kDfmTableSize))) return r;
  if ((r = cuda_check(c, cudaMemcpyAsync(c->dfm, tab.data(), sizeof(float2) * kDfmTableSize, cudaMemcpyHostToDevice,
                                         c->stream),
                      "function table upload")))
    return r;
  return cuda_check(c, cudaStreamSynchronize(c->stream), "function table upload");
}

void launch_pair_build(amp_ctx* c) {
  // the split multipoles also feed the float64 path's reciprocal spreading,
  // so they are made even when there are no pairs
  c->n_launch += 1;
  k_split_multipoles<<<amp_blocks(c->n, 256), 256, 0, c->stream>>>(c->n, c->atomA, c->atomB, c->atomC, c->atomD,
                                                                  c->mp_df, c->pd, c->xhl);
  if (c->cfg.precision == AMP_FP64) cudaMemsetAsync(c->e0intra, 0, sizeof(double4_32a) * c->n, c->stream);
  if (c->n_half == 0) return;
  const PairGeom g = geom(c);
  const int blocks = amp_blocks(c->n_half, 256);
  c->n_launch += 1;
  if (c->cfg.precision == AMP_FP64) {
    const PairGeomDf gd = geom_df(g);
    cudaMemsetAsync(c->intra, 0, sizeof(int), c->stream);
    k_pair_build_df<<<blocks, 256, 0, c->stream>>>(c->n_half, c->half_i, c->half_j, c->pd, c->mp_df, gd, c->dfm,
                                                   c->full_start, c->half_start, c->pos_tr, c->C64,
                                                   reinterpret_cast<float*>(c->Ep64), c->intra);
    c->n_launch += 1;
    k_intra_fields64<<<4 * c->n_sm, 128, 0, c->stream>>>(c->intra, c->half_i, c->half_j, g, c->atomA, c->atomB,
                                                         c->atomC, c->atomD, c->e0intra);
    return;
  }
  // mixed path: float32 pair terms from the split records, which also serve its float64 check
  PairGeom32 g32;
  g32.beta = (float)g.beta;
  g32.twob2 = (float)g.twob2;
  g32.gpre = (float)g.gpre;
  cudaMemsetAsync(c->intra, 0, sizeof(int), c->stream);
  k_pair_build32<<<blocks, 256, 0, c->stream>>>(c->n_half, c->half_i, c->half_j, c->pd, c->mp_df, geom_df(g), g32,
                                                c->full_start, c->half_start, c->pos_tr,
                                                reinterpret_cast<float4*>(c->T32),
                                                reinterpret_cast<float2*>(c->T32 + 4 * c->cap_full), c->Ep32,
                                                c->intra);
}

// The split positions and moments alone (clusters, which build no pair terms).
// out += (the permanent field with scale s for two sites of one molecule) -
// (that with scale 0); periodic contexts (the pair build's intramolecular list).
void launch_intra_scaled(amp_ctx* c, double s, double4_32a* out) {
  if (c->n_half == 0) return;
  c->n_launch += 1;
  k_intra_scaled64<<<4 * c->n_sm, 128, 0, c->stream>>>(c->intra, c->half_i, c->half_j, geom(c), s, c->atomA,
                                                       c->atomB, c->atomC, c->atomD, out);
}

void launch_split_multipoles(amp_ctx* c) {
  c->n_launch += 1;
  k_split_multipoles<<<amp_blocks(c->n, 256), 256, 0, c->stream>>>(c->n, c->atomA, c->atomB, c->atomC, c->atomD,
                                                                  c->mp_df, c->pd, c->xhl);
}

// Real-space permanent field with the self term +4 beta^3/(3 sqrt(pi)) d_i (d_i from atomB).
void launch_e0_real(amp_ctx* c, double4_32a* out) {
  const PairGeom g = geom(c);
  const int blocks = amp_blocks((long long)c->n * kRowGroup, 256);
  c->n_launch += 1;
  if (c->cfg.precision == AMP_FP64)
    k_row_sum_fields_df<<<blocks, 256, 0, c->stream>>>(c->n, c->full_start, c->full_ref,
                                                       reinterpret_cast<const float*>(c->Ep64), g.selfc, c->atomB,
                                                       c->e0intra, out);
  else
    k_row_sum_pairvec<float><<<blocks, 256, 0, c->stream>>>(c->n, c->full_start, c->full_ref, c->Ep32, g.selfc,
                                                            c->atomB, out);
}

// v must be mirrored in its float-pair split, which the kernel reads from vhl
// (every split kernel writes it beside p32 / plo).
void launch_t_real(amp_ctx* c, const double4_32a* v, double4_32a* out) {
  const PairGeom g = geom(c);
  c->n_launch += 1;
  const int tb = (int)std::min<long long>(amp_blocks((long long)c->n * kRowGroup, 256),
                                          (long long)kTRealBlocksPerSmDf * c->n_sm);
  k_t_real_df<<<tb, 256, 0, c->stream>>>(c->n, c->full_start, c->full_j, c->C64, c->xhl, geom_df(g), g.selfc,
                                         c->vhl, v, out, c->op_stop);
}

void launch_t_real32(amp_ctx* c, const float4* v32, const double4_32a* v64, double4_32a* out) {
  const PairGeom g = geom(c);
  c->n_launch += 1;
  const int tb = (int)std::min<long long>(amp_blocks((long long)c->n * kRowGroup, 256),
                                          (long long)kTRealBlocksPerSm32 * c->n_sm);
  k_t_real32<<<tb, 256, 0, c->stream>>>(c->n, c->full_start, c->full_j, reinterpret_cast<const float4*>(c->T32),
                                        reinterpret_cast<const float2*>(c->T32 + 4 * c->cap_full), g.selfc, v32, v64,
                                        out, c->op_stop);
}

// v's split must be in p32/plo (free during the check: k_cg_init rewrites
// them); the caller splits it before the reciprocal part forks.
void launch_t_real_fp64_direct(amp_ctx* c, const double4_32a* v, double4_32a* out) {
  const PairGeom g = geom(c);
  const int blocks = amp_blocks((long long)c->n * kRowGroup, 256);
  c->n_launch += c->n_half > 0 ? 2 : 1;
  if (c->n_half > 0)
    k_pair_tv_df<<<amp_blocks(c->n_half, 256), 256, 0, c->stream>>>(c->n_half, c->half_i, c->half_j, c->pd,
                                                                    geom_df(g), c->dfm, c->p32, c->plo,
                                                                    reinterpret_cast<float*>(c->Ep64));
  k_row_sum_fields_df<<<blocks, 256, 0, c->stream>>>(c->n, c->full_start, c->full_ref,
                                                     reinterpret_cast<const float*>(c->Ep64), g.selfc, v, nullptr,
                                                     out);
}

}  // namespace amp
