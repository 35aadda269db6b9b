// Isolated clusters (no periodic box): every pair interacts, no cutoff, no
// Ewald screening (beta = 0), no reciprocal or self terms. The kernels are
// then B1 = 1/r^3, B2 = 3/r^5, B3 = 15/r^7 with Thole damping, and the
// permanent field skips pairs inside one molecule (their damped kernel
// B_n - bare_n vanishes when beta = 0).
//
// All-pairs tiles: a block owns kTileI rows and one slice of the columns
// (blockIdx.y); the column slice is staged through shared memory tile by
// tile. Each thread sums a tile in the working precision R and adds the tile
// sum to float64 accumulators. Slices are summed by a second kernel in a
// fixed order (no atomics), so results do not depend on scheduling.
#include "amp_internal.cuh"

namespace amp {
namespace {

constexpr int kTileI = 64;  // rows per block (threads)
constexpr int kTileJ = 64;  // columns staged per shared-memory tile

template <typename R>
struct JTile {
  R x[kTileJ], y[kTileJ], z[kTileJ], isa[kTileJ], th[kTileJ];
  int mol[kTileJ];
  R v[kTileJ][3];      // dipoles (T*v) or permanent dipoles
  R q[kTileJ];
  R quad[kTileJ][6];
};

template <typename R, bool kPerm, typename V>
__global__ void __launch_bounds__(kTileI) k_cluster_field(int n, int cols_per_slice, const double4_32a* __restrict__ A,
                                                          const double4_32a* __restrict__ B,
                                                          const double4_32a* __restrict__ C,
                                                          const double4_32a* __restrict__ D, const V* __restrict__ v,
                                                          double4_32a* __restrict__ part,
                                                          const int* __restrict__ stop) {
  if (stop && *stop) return;
  __shared__ JTile<R> t;
  const int i = blockIdx.x * kTileI + threadIdx.x;
  const int j0 = blockIdx.y * cols_per_slice;
  const int j1 = min(n, j0 + cols_per_slice);
  R xi = 0, yi = 0, zi = 0, isai = 0, thi = 0;
  int moli = -1;
  if (i < n) {
    const double4_32a a = A[i], b = B[i], d = D[i];
    xi = (R)a.x;
    yi = (R)a.y;
    zi = (R)a.z;
    isai = (R)b.w;
    thi = (R)d.z;
    moli = (int)d.w;
  }
  double ax = 0.0, ay = 0.0, az = 0.0;
  for (int jt = j0; jt < j1; jt += kTileJ) {
    const int jl = jt + threadIdx.x;
    if (threadIdx.x < kTileJ && jl < j1) {
      const double4_32a a = A[jl], b = B[jl], d = D[jl];
      t.x[threadIdx.x] = (R)a.x;
      t.y[threadIdx.x] = (R)a.y;
      t.z[threadIdx.x] = (R)a.z;
      t.isa[threadIdx.x] = (R)b.w;
      t.th[threadIdx.x] = (R)d.z;
      t.mol[threadIdx.x] = (int)d.w;
      if (kPerm) {
        const double4_32a c = C[jl];
        t.q[threadIdx.x] = (R)a.w;
        t.v[threadIdx.x][0] = (R)b.x;
        t.v[threadIdx.x][1] = (R)b.y;
        t.v[threadIdx.x][2] = (R)b.z;
        t.quad[threadIdx.x][0] = (R)c.x;
        t.quad[threadIdx.x][1] = (R)c.y;
        t.quad[threadIdx.x][2] = (R)c.z;
        t.quad[threadIdx.x][3] = (R)c.w;
        t.quad[threadIdx.x][4] = (R)d.x;
        t.quad[threadIdx.x][5] = (R)d.y;
      } else {
        const V m = v[jl];
        t.v[threadIdx.x][0] = (R)m.x;
        t.v[threadIdx.x][1] = (R)m.y;
        t.v[threadIdx.x][2] = (R)m.z;
      }
    }
    __syncthreads();
    const int cnt = min(kTileJ, j1 - jt);
    R sx = 0, sy = 0, sz = 0;
    if (i < n) {
      for (int k = 0; k < cnt; ++k) {
        const int j = jt + k;
        if (j == i) continue;
        if (kPerm && t.mol[k] == moli) continue;  // excluded: damped kernel vanishes
        const R rx = xi - t.x[k], ry = yi - t.y[k], rz = zi - t.z[k];
        const R r2 = rx * rx + ry * ry + rz * rz;
        const R ir = (R)1 / sqrt(r2);
        const R ir2 = ir * ir;
        const R x = min(thi, t.th[k]) * r2 * sqrt(r2) * isai * t.isa[k];
        const R e = exp(-x);
        const R b1 = ((R)1 - e) * ir * ir2;
        const R b2 = (R)3 * ((R)1 - ((R)1 + x) * e) * ir2 * ir2 * ir;
        if (kPerm) {
          const R b3 = (R)15 * ((R)1 - ((R)1 + x + (R)0.6 * x * x) * e) * ir2 * ir2 * ir2 * ir;
          const R* Q = t.quad[k];
          const R tx = Q[0] * rx + Q[3] * ry + Q[4] * rz;
          const R ty = Q[3] * rx + Q[1] * ry + Q[5] * rz;
          const R tz = Q[4] * rx + Q[5] * ry + Q[2] * rz;
          const R rtr = rx * tx + ry * ty + rz * tz;
          const R dr = t.v[k][0] * rx + t.v[k][1] * ry + t.v[k][2] * rz;
          const R rad = t.q[k] * b1 + b2 * dr + b3 * rtr * (R)(1.0 / 3.0);
          const R c2 = b2 * (R)(2.0 / 3.0);
          sx += rad * rx - b1 * t.v[k][0] - c2 * tx;
          sy += rad * ry - b1 * t.v[k][1] - c2 * ty;
          sz += rad * rz - b1 * t.v[k][2] - c2 * tz;
        } else {
          const R s = b2 * (t.v[k][0] * rx + t.v[k][1] * ry + t.v[k][2] * rz);
          sx += s * rx - b1 * t.v[k][0];
          sy += s * ry - b1 * t.v[k][1];
          sz += s * rz - b1 * t.v[k][2];
        }
      }
    }
    ax += (double)sx;
    ay += (double)sy;
    az += (double)sz;
    __syncthreads();
  }
  if (i < n) part[(long long)blockIdx.y * n + i] = make_double4_32a(ax, ay, az, 0.0);
}

// The float64 path of the same sums in double-float (hi + lo floats, float
// units only): positions, moments and v are split as they are staged, the
// kernels and the Thole exponential come from df_rsqrt / df_exp_neg, and each
// thread keeps its row sum in double-float across all tiles.
struct JTileDf {
  float xh[kTileJ], xl[kTileJ], yh[kTileJ], yl[kTileJ], zh[kTileJ], zl[kTileJ];
  float ish[kTileJ], isl[kTileJ], thh[kTileJ], thl[kTileJ];
  int mol[kTileJ];
  float mp[kTileJ][20];  // v (or q, d, Theta) as hi/lo pairs in the order of mp_field_df
};

__device__ __forceinline__ dflt df_min(dflt a, dflt b) { return (a.hi < b.hi || (a.hi == b.hi && a.lo <= b.lo)) ? a : b; }

template <bool kPerm>
__global__ void __launch_bounds__(kTileI) k_cluster_field_df(int n, int cols_per_slice,
                                                             const double4_32a* __restrict__ A,
                                                             const double4_32a* __restrict__ B,
                                                             const double4_32a* __restrict__ C,
                                                             const double4_32a* __restrict__ D,
                                                             const double4_32a* __restrict__ v,
                                                             const float2* __restrict__ tab,
                                                             double4_32a* __restrict__ part,
                                                             const int* __restrict__ stop) {
  if (stop && *stop) return;
  __shared__ JTileDf t;
  const int i = blockIdx.x * kTileI + threadIdx.x;
  const int j0 = blockIdx.y * cols_per_slice;
  const int j1 = min(n, j0 + cols_per_slice);
  dflt xi = {0.f, 0.f}, yi = xi, zi = xi, isai = xi, thi = xi;
  int moli = -1;
  if (i < n) {
    const double4_32a a = A[i], b = B[i], d = D[i];
    xi = df_split(a.x);
    yi = df_split(a.y);
    zi = df_split(a.z);
    isai = df_split(b.w);
    thi = df_split(d.z);
    moli = (int)d.w;
  }
  const dflt ONE = {1.f, 0.f}, THREE = {3.f, 0.f}, FIFTEEN = {15.f, 0.f};
  const dflt six = {0.600000024f, -2.38418579e-08f};  // 0.6 = hi + lo
  dflt sx = {0.f, 0.f}, sy = sx, sz = sx;
  for (int jt = j0; jt < j1; jt += kTileJ) {
    const int jl = jt + threadIdx.x;
    if (threadIdx.x < kTileJ && jl < j1) {
      const double4_32a a = A[jl], b = B[jl], d = D[jl];
      dflt u = df_split(a.x);
      t.xh[threadIdx.x] = u.hi, t.xl[threadIdx.x] = u.lo;
      u = df_split(a.y);
      t.yh[threadIdx.x] = u.hi, t.yl[threadIdx.x] = u.lo;
      u = df_split(a.z);
      t.zh[threadIdx.x] = u.hi, t.zl[threadIdx.x] = u.lo;
      u = df_split(b.w);
      t.ish[threadIdx.x] = u.hi, t.isl[threadIdx.x] = u.lo;
      u = df_split(d.z);
      t.thh[threadIdx.x] = u.hi, t.thl[threadIdx.x] = u.lo;
      t.mol[threadIdx.x] = (int)d.w;
      float* m = t.mp[threadIdx.x];
      if (kPerm) {
        const double4_32a c = C[jl];
        const double vals[10] = {a.w, b.x, b.y, b.z, c.x, c.y, c.z, c.w, d.x, d.y};
        for (int k = 0; k < 10; ++k) {
          const dflt w = df_split(vals[k]);
          m[2 * k] = w.hi;
          m[2 * k + 1] = w.lo;
        }
      } else {
        const double4_32a vv = v[jl];
        const double vals[3] = {vv.x, vv.y, vv.z};
        for (int k = 0; k < 3; ++k) {
          const dflt w = df_split(vals[k]);
          m[2 * k] = w.hi;
          m[2 * k + 1] = w.lo;
        }
      }
    }
    __syncthreads();
    const int cnt = min(kTileJ, j1 - jt);
    if (i < n) {
      for (int k = 0; k < cnt; ++k) {
        const int j = jt + k;
        if (j == i) continue;
        if (kPerm && t.mol[k] == moli) continue;  // excluded: damped kernel vanishes
        const dflt R[3] = {df_sub(xi, {t.xh[k], t.xl[k]}), df_sub(yi, {t.yh[k], t.yl[k]}),
                           df_sub(zi, {t.zh[k], t.zl[k]})};
        const dflt r2 = df_madd(R[2], R[2], df_madd(R[1], R[1], df_mul(R[0], R[0])));
        const dflt ir = df_rsqrt(r2);
        const dflt ir2 = df_mul(ir, ir);
        const dflt x = df_mul(df_mul(df_min(thi, {t.thh[k], t.thl[k]}), df_mul(r2, df_mul(r2, ir))),
                              df_mul(isai, {t.ish[k], t.isl[k]}));
        const dflt e = df_exp_neg(x, tab);
        const dflt ir3 = df_mul(ir, ir2), ir5 = df_mul(ir3, ir2);
        const dflt b1 = df_mul(df_sub(ONE, e), ir3);
        const dflt b2 = df_mul(df_mul(THREE, df_sub(ONE, df_mul(df_add(ONE, x), e))), ir5);
        const float* m = t.mp[k];
        if (kPerm) {
          const dflt x1 = df_add(ONE, x);
          const dflt b3 = df_mul(df_mul(FIFTEEN, df_sub(ONE, df_mul(df_madd(df_mul(six, x), x, x1), e))),
                                 df_mul(ir5, ir2));
          dflt mp[10];
          for (int q = 0; q < 10; ++q) mp[q] = {m[2 * q], m[2 * q + 1]};
          dflt f[3];
          mp_field_df(R, mp, b1, b2, b3, f);
          sx = df_add(sx, f[0]);
          sy = df_add(sy, f[1]);
          sz = df_add(sz, f[2]);
        } else {
          const dflt vx = {m[0], m[1]}, vy = {m[2], m[3]}, vz = {m[4], m[5]};
          const dflt s = df_mul(b2, df_madd(R[2], vz, df_madd(R[1], vy, df_mul(R[0], vx))));
          sx = df_add(sx, df_sub(df_mul(s, R[0]), df_mul(b1, vx)));
          sy = df_add(sy, df_sub(df_mul(s, R[1]), df_mul(b1, vy)));
          sz = df_add(sz, df_sub(df_mul(s, R[2]), df_mul(b1, vz)));
        }
      }
    }
    __syncthreads();
  }
  if (i < n)
    part[(long long)blockIdx.y * n + i] = make_double4_32a(df_to_double(sx), df_to_double(sy), df_to_double(sz), 0.0);
}

// The mixed path's T*v over all pairs in float32: positions, 1/sqrt(alpha),
// Thole a and molecule as float records (clu32, made once per geometry), v
// as floats, so the tiles are staged without float64 conversions. A full
// tile without the row's own atom runs an unrolled loop with no self test
// (the kernel is bound by instruction issue: T*v of a 12,288-atom cluster
// 0.272 against 0.319 ms with the tested loop everywhere).
struct JTile32 {
  float4 p[kTileJ];  // x, y, z, 1/sqrt(alpha)
  float th[kTileJ];
  float4 v[kTileJ];
};

// One pair's term T_ij v_j of the float32 all-pairs product, added to (sx, sy, sz).
__device__ __forceinline__ void tv32_pair(const float4& pi, float thi, const float4& pj, float thj, const float4& vj,
                                          float& sx, float& sy, float& sz) {
  const float rx = pi.x - pj.x, ry = pi.y - pj.y, rz = pi.z - pj.z;
  const float r2 = rx * rx + ry * ry + rz * rz;
  const float ir = rsqrtf(r2);
  const float ir2 = ir * ir;
  const float x = fminf(thi, thj) * r2 * r2 * ir * pi.w * pj.w;
  const float e = expf(-x);
  const float b1 = (1.f - e) * ir * ir2;
  const float b2 = 3.f * (1.f - (1.f + x) * e) * ir2 * ir2 * ir;
  const float sv = b2 * (vj.x * rx + vj.y * ry + vj.z * rz);
  sx += sv * rx - b1 * vj.x;
  sy += sv * ry - b1 * vj.y;
  sz += sv * rz - b1 * vj.z;
}

__global__ void __launch_bounds__(kTileI) k_cluster_tv32(int n, int cols_per_slice, const float4* __restrict__ clu32,
                                                         const float4* __restrict__ v32,
                                                         double4_32a* __restrict__ part,
                                                         const int* __restrict__ stop) {
  if (stop && *stop) return;
  __shared__ JTile32 t;
  const int i = blockIdx.x * kTileI + threadIdx.x;
  const int j0 = blockIdx.y * cols_per_slice;
  const int j1 = min(n, j0 + cols_per_slice);
  float4 pi = make_float4(0.f, 0.f, 0.f, 0.f);
  float thi = 0.f;
  if (i < n) {
    pi = clu32[2 * (long long)i];
    thi = clu32[2 * (long long)i + 1].x;
  }
  double ax = 0.0, ay = 0.0, az = 0.0;
  for (int jt = j0; jt < j1; jt += kTileJ) {
    const int jl = jt + threadIdx.x;
    if (threadIdx.x < kTileJ && jl < j1) {
      t.p[threadIdx.x] = clu32[2 * (long long)jl];
      t.th[threadIdx.x] = clu32[2 * (long long)jl + 1].x;
      t.v[threadIdx.x] = v32[jl];
    }
    __syncthreads();
    const int cnt = min(kTileJ, j1 - jt);
    float sx = 0.f, sy = 0.f, sz = 0.f;
    if (i < n) {
      if (cnt == kTileJ && (i < jt || i >= jt + kTileJ)) {  // a full tile without the row's own atom
#pragma unroll 8
        for (int k = 0; k < kTileJ; ++k) tv32_pair(pi, thi, t.p[k], t.th[k], t.v[k], sx, sy, sz);
      } else {
        for (int k = 0; k < cnt; ++k)
          if (jt + k != i) tv32_pair(pi, thi, t.p[k], t.th[k], t.v[k], sx, sy, sz);
      }
    }
    ax += (double)sx;
    ay += (double)sy;
    az += (double)sz;
    __syncthreads();
  }
  if (i < n) part[(long long)blockIdx.y * n + i] = make_double4_32a(ax, ay, az, 0.0);
}

__global__ void k_cluster_records32(int n, const double4_32a* __restrict__ A, const double4_32a* __restrict__ B,
                                    const double4_32a* __restrict__ D, float4* __restrict__ clu32) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double4_32a a = A[i], b = B[i], d = D[i];
  clu32[2 * (long long)i] = make_float4((float)a.x, (float)a.y, (float)a.z, (float)b.w);
  clu32[2 * (long long)i + 1] = make_float4((float)d.z, 0.f, 0.f, 0.f);
}

__global__ void k_cluster_reduce(int n, int slices, const double4_32a* __restrict__ part, double4_32a* __restrict__ out,
                                 const int* __restrict__ stop) {
  if (stop && *stop) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double x = 0, y = 0, z = 0;
  for (int s = 0; s < slices; ++s) {
    const double4_32a p = part[(long long)s * n + i];
    x += p.x;
    y += p.y;
    z += p.z;
  }
  out[i] = make_double4_32a(x, y, z, 0.0);
}

__global__ void k_identity_perm(int n, int* __restrict__ perm) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) perm[i] = i;
}

__global__ void k_cluster_atoms(int n, const double* __restrict__ xyz, const double* __restrict__ q,
                                const double* __restrict__ dip, const double* __restrict__ quad,
                                const double* __restrict__ alpha, const double* __restrict__ thole,
                                const int* __restrict__ mol, double4_32a* __restrict__ A, double4_32a* __restrict__ B,
                                double4_32a* __restrict__ C, double4_32a* __restrict__ D, double2* __restrict__ alph,
                                int* __restrict__ flags) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double al = alpha[i];
  if (!(al > 0.0)) atomicOr(&flags[0], 2);
  alph[i] = make_double2(al, 1.0 / al);
  A[i] = make_double4_32a(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], q[i]);
  B[i] = make_double4_32a(dip[3 * i], dip[3 * i + 1], dip[3 * i + 2], 1.0 / sqrt(al));
  C[i] = make_double4_32a(quad[6 * i], quad[6 * i + 1], quad[6 * i + 2], quad[6 * i + 3]);
  D[i] = make_double4_32a(quad[6 * i + 4], quad[6 * i + 5], thole[i], (double)mol[i]);
}

// Column slices so that the grid covers about 32 blocks of 64 threads per
// SM of the 152: 1024 threads, whose latency-bound pair loops (rsqrt, exp and
// the dependent multiply-adds) then keep each SM busy. Against 2 blocks per
// SM: the 4,096-water cluster's solve 6.1 vs 12.4 ms (mixed) and 25.4 vs
// 43.5 ms (float64); 8, 16 and 64 blocks gave 7.2, 6.6 and 5.9 ms (mixed).
int slices_for(int n) {
  const int rows = (n + kTileI - 1) / kTileI;
  int s = (32 * 152 + rows - 1) / rows;
  const int max_s = (n + kTileJ - 1) / kTileJ;
  if (s > max_s) s = max_s;
  if (s > kClusterMaxSlices) s = kClusterMaxSlices;
  return s < 1 ? 1 : s;
}

template <bool kPerm, typename R, typename V>
void launch_field(amp_ctx* c, const V* v, double4_32a* out) {
  const int n = c->n;
  const int s = slices_for(n);
  int cols = (n + s - 1) / s;
  cols = (cols + kTileJ - 1) / kTileJ * kTileJ;
  dim3 grid((n + kTileI - 1) / kTileI, s);
  c->n_launch += 2;
  if constexpr (sizeof(R) == 8)  // float64 path: double-float arithmetic
    k_cluster_field_df<kPerm><<<grid, kTileI, 0, c->stream>>>(n, cols, c->atomA, c->atomB, c->atomC, c->atomD,
                                                               reinterpret_cast<const double4_32a*>(v), c->dfm,
                                                               c->cluster_part, c->op_stop);
  else if constexpr (!kPerm)
    k_cluster_tv32<<<grid, kTileI, 0, c->stream>>>(n, cols, c->clu32, reinterpret_cast<const float4*>(v),
                                                    c->cluster_part, c->op_stop);
  else
    k_cluster_field<R, kPerm, V><<<grid, kTileI, 0, c->stream>>>(n, cols, c->atomA, c->atomB, c->atomC, c->atomD,
                                                                  v, c->cluster_part, c->op_stop);
  k_cluster_reduce<<<amp_blocks(n, 256), 256, 0, c->stream>>>(n, s, c->cluster_part, out, c->op_stop);
}

}  // namespace

int cluster_setup(amp_ctx* c, const double* xyz, const double* q, const double* dip, const double* quad,
                  const double* alpha, const double* thole, const int* mol) {
  const int n = c->n;
  cudaStream_t st = c->stream;
  int r;
  if (c->cluster_part_cap < (long long)kClusterMaxSlices * n) {
    dev_free(c, c->cluster_part);
    c->cluster_part = nullptr;
    if ((r = dev_alloc(c, &c->cluster_part, (long long)kClusterMaxSlices * n))) return r;
    c->cluster_part_cap = (long long)kClusterMaxSlices * n;
  }
  if (c->cfg.precision == AMP_MIXED && c->clu32_cap < n) {
    dev_free(c, c->clu32);
    c->clu32 = nullptr;
    if ((r = dev_alloc(c, &c->clu32, 2LL * n))) return r;
    c->clu32_cap = n;
  }
  cudaMemsetAsync(c->flags, 0, sizeof(int) * 4, st);
  c->n_launch += 2;
  k_identity_perm<<<amp_blocks(n, 256), 256, 0, st>>>(n, c->perm);
  k_cluster_atoms<<<amp_blocks(n, 256), 256, 0, st>>>(n, xyz, q, dip, quad, alpha, thole, mol, c->atomA, c->atomB,
                                                      c->atomC, c->atomD, c->alph, c->flags);
  if (c->clu32) {
    c->n_launch += 1;
    k_cluster_records32<<<amp_blocks(n, 256), 256, 0, st>>>(n, c->atomA, c->atomB, c->atomD, c->clu32);
  }
  cudaMemcpyAsync(&c->hibuf[2], c->flags, sizeof(int), cudaMemcpyDeviceToHost, st);
  if ((r = cuda_check(c, cudaStreamSynchronize(st), "cluster setup"))) return r;
  if (c->hibuf[2] & 2) return fail(c, AMP_ERR_ARG, "alpha must be > 0 for every site");
  c->n_half = (long long)n * (n - 1) / 2;
  c->n_full = 2 * c->n_half;
  return AMP_OK;
}

void cluster_permanent_field(amp_ctx* c, double4_32a* out) {
  if (c->cfg.precision == AMP_FP64)
    launch_field<true, double, double4_32a>(c, (const double4_32a*)nullptr, out);
  else
    launch_field<true, float, double4_32a>(c, (const double4_32a*)nullptr, out);
}

void cluster_t(amp_ctx* c, const double4_32a* v, const float4* v32, double4_32a* out, bool fp64) {
  if (fp64)
    launch_field<false, double, double4_32a>(c, v, out);
  else
    launch_field<false, float, float4>(c, v32, out);
}

}  // namespace amp
