// Batched solves of many small isolated clusters (the serving path's device
// engine; the paper has no serving counterpart: its throughput runs are many
// MPI ranks on one system, Section "Parallel performance").
//
// Every admitted cluster owns a tile-aligned range of one device arena and a
// request slot with its PCG state. One iteration of every request in flight
// is two launches of persistent kernels, each of which pulls
// (request, 64-row tile) work items from a device queue (an item list and an
// atomic head) until the list is exhausted:
//   T (pair phase): all-pairs sums over the request's atoms for the tile's
//     rows, the columns staged through shared memory: the permanent field
//     E0, the product T*v in float32 (v the float32 copy of the dipoles), or
//     the float64 check T*mu in double-float; the row sums are kept in
//     double-float, the epilogue in float64;
//   S (vector phase): the PCG vector update of the tile's atoms from the
//     request's reduced partial sums, in float64.
// Requests of any size share the launches; each request's sums are taken in a
// fixed order (tile partials reduced in tile order), so a request's result
// does not depend on what else is in flight.
//
// The solver is the diagonal-preconditioned CG of amp_pcg.cu in the same
// Chronopoulos-Gear arrangement (the operator applied to z, w = A z; rho =
// r.z, m = z.w; beta = rho/rho_old; gamma = rho/(m - beta rho/gamma_old);
// p = z + beta p; q = w + beta q; mu += gamma p; r -= gamma q; z = alpha r),
// started from mu = alpha E0, stopped when 4.8032047 sqrt(sum |z_i|^2 / N)
// < tol. Mixed precision: float32 pair terms, float64 sums and scalars; when
// the float32 iteration has converged, the residual is recomputed with the
// pair terms in double-float, and the iteration continues from it (restart,
// beta = 0) unless it is below tol too.
//
// A request's state moves between the two kernels through two records, each
// written by tile 0 of one kernel and read by every tile of the other:
//   ReqT (written by S, read by T): what T does next, iteration, scalars;
//   ReqS (written by T, read by S): what S does next, the scalars it needs.
// No kernel waits on another: the launches' order on one stream is the only
// synchronisation.
#include <algorithm>
#include <vector>

#include "amp_internal.cuh"
#include "amp_batch.cuh"

namespace amp {
namespace batch {

using ::amp::dflt;

// ---------------------------------------------------------------- kernels

__device__ __forceinline__ void acc_add(dflt& acc, float x) {  // acc += x, error-free two-sum
  const dflt s = df_two_sum(acc.hi, x);
  acc.hi = s.hi;
  acc.lo = __fadd_rn(acc.lo, s.lo);
}

// One work item per CTA iteration; thread 0 takes it from the queue.
__device__ __forceinline__ int next_item(int* head) {
  __shared__ int item;
  __syncthreads();
  if (threadIdx.x == 0) item = atomicAdd(head, 1);
  __syncthreads();
  return item;
}

// Sum of a double over the block (kThreads), valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < kThreads / 32; ++w) s += red[w];
  return s;
}

// Sum of nt partials in tile order (one warp), broadcast.
__device__ __forceinline__ double reduce_tiles(const double* __restrict__ part, int t0, int nt, double* bc) {
  __syncthreads();
  if (threadIdx.x < 32) {
    double s = 0.0;
    for (int k = threadIdx.x; k < nt; k += 32) s += __ldcg(part + t0 + k);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) *bc = s;
  }
  __syncthreads();
  return *bc;
}

struct Stage {
  float4 a[kChunk];   // TV/E0: (x, y, z, 1/sqrt(alpha)); check: hi parts
  float4 b[kChunk];   // TV: v; E0: (q, dx, dy, dz); check: lo parts
  float4 c[kChunk];   // E0: (Qxx, Qyy, Qzz, Qxy); check: (thole hi, lo, molecule, 0)
  float4 d[kChunk];   // E0: (Qxz, Qyz, thole, molecule); check: mu hi
  float4 e[kChunk];   // check: mu lo; TV: (thole, molecule, 0, 0)
};

// Float32 pair kernels of a cluster pair (beta = 0) with Thole damping:
// x = a r^3/sqrt(alpha_i alpha_j), b1 = (1 - e^-x)/r^3,
// b2 = 3 (1 - (1 + x) e^-x)/r^5, b3 = 15 (1 - (1 + x + 0.6 x^2) e^-x)/r^7.
__device__ __forceinline__ void thole32(float r2, float a, float isa, float& b1, float& b2, float& b3, bool want3) {
  const float ir = rsqrtf(r2), ir2 = ir * ir, ir3 = ir * ir2;
  const float x = a * r2 * (r2 * ir) * isa;
  const float e = expf(-x);
  b1 = (1.f - e) * ir3;
  b2 = 3.f * (1.f - (1.f + x) * e) * ir3 * ir2;
  b3 = want3 ? 15.f * (1.f - (1.f + x + 0.6f * x * x) * e) * ir3 * ir2 * ir2 : 0.f;
}

__device__ __forceinline__ dflt df_min2(dflt a, dflt b) { return (a.hi < b.hi || (a.hi == b.hi && a.lo <= b.lo)) ? a : b; }

__global__ void __launch_bounds__(kThreads) k_batch_pairs(Arena A, int n_items, const int2* __restrict__ items,
                                                          int* __restrict__ heads, const float2* __restrict__ tab) {
  __shared__ Stage st;
  __shared__ double red[kThreads / 32];
  __shared__ double bc;
  if (blockIdx.x == 0 && threadIdx.x == 0) heads[1] = 0;  // the vector phase's queue, for the next launch
  const int row = threadIdx.x >> 1, h = threadIdx.x & 1;
  while (true) {
    const int it = next_item(heads);
    if (it >= n_items) break;
    const int2 w = items[it];
    const int rq = w.x, tile = w.y;
    const ReqInfo info = A.info[rq];
    const ReqT rt = A.reqT[rq];
    // ---- what this request does in this launch (every tile decides alike)
    int act = A_IDLE;
    double rms = 0.0;
    if (rt.kind == K_E0) {
      act = A_E0;
    } else if (rt.kind == K_INIT) {
      act = A_TV;
    } else if (rt.kind == K_ITER || rt.kind == K_AFTER) {
      const double zz = reduce_tiles(A.partz, info.tile0, info.ntiles, &bc);
      rms = kDebye * sqrt(zz / (double)info.n);
      if (rms < info.tol)
        act = rt.kind == K_ITER ? A_CHECK : A_FINISH;
      else if (rt.iter >= info.max_iter)
        act = A_FINISH;
      else
        act = A_TVI;
    }
    if (tile == 0 && threadIdx.x == 0) {
      ReqS s;
      s.act = act;
      s.iter = rt.iter;
      s.first = rt.first;
      s.rho_old = rt.rho;
      s.gamma_old = rt.gamma;
      s.rms = rms;
      A.reqS[rq] = s;  // an idle request's record tells the vector phase to skip it
    }
    if (act == A_IDLE) continue;
    if (act == A_FINISH) {
      const double e = reduce_tiles(A.parte, info.tile0, info.ntiles, &bc);
      if (tile == 0 && threadIdx.x == 0) {
        ReqOut o;
        o.status = rms < info.tol ? 1 : 2;
        o.iters = rt.iter;
        o.rms = rms;
        o.U = -0.5 * kCoulomb * e;
        A.out[rq] = o;
      }
      continue;
    }
    // ---- pair sums for the tile's rows, columns staged through shared memory
    const int il = tile * kRows + row;  // row within the request
    const bool valid = il < info.n;
    const int gi = info.off + (valid ? il : 0);
    dflt sx = {0.f, 0.f}, sy = sx, sz = sx;
    if (act == A_CHECK) {
      const float4 ph = A.pdf[3 * (long long)gi], pl = A.pdf[3 * (long long)gi + 1], pt = A.pdf[3 * (long long)gi + 2];
      const dflt xi = {ph.x, pl.x}, yi = {ph.y, pl.y}, zi = {ph.z, pl.z}, isai = {ph.w, pl.w}, thi = {pt.x, pt.y};
      const dflt ONE = {1.f, 0.f}, THREE = {3.f, 0.f};
      for (int j0 = 0; j0 < info.n; j0 += kChunk) {
        __syncthreads();
        const int jl = j0 + threadIdx.x;
        if (jl < info.n) {
          const long long g = info.off + jl;
          st.a[threadIdx.x] = A.pdf[3 * g];
          st.b[threadIdx.x] = A.pdf[3 * g + 1];
          st.c[threadIdx.x] = A.pdf[3 * g + 2];
          const double4_32a m = A.mu[g];
          const dflt mx = df_split(m.x), my = df_split(m.y), mz = df_split(m.z);
          st.d[threadIdx.x] = make_float4(mx.hi, my.hi, mz.hi, 0.f);
          st.e[threadIdx.x] = make_float4(mx.lo, my.lo, mz.lo, 0.f);
        }
        __syncthreads();
        const int cnt = min(kChunk, info.n - j0);
        if (valid)
          for (int k = h; k < cnt; k += 2) {
            if (j0 + k == il) continue;
            const float4 jh = st.a[k], jlo = st.b[k], jt = st.c[k], vh = st.d[k], vl = st.e[k];
            const dflt R[3] = {df_sub(xi, {jh.x, jlo.x}), df_sub(yi, {jh.y, jlo.y}), df_sub(zi, {jh.z, jlo.z})};
            const dflt r2 = df_madd(R[2], R[2], df_madd(R[1], R[1], df_mul(R[0], R[0])));
            const dflt ir = df_rsqrt(r2);
            const dflt ir2 = df_mul(ir, ir);
            const dflt x = df_mul(df_mul(df_min2(thi, {jt.x, jt.y}), df_mul(r2, df_mul(r2, ir))),
                                  df_mul(isai, {jh.w, jlo.w}));
            const dflt e = df_exp_neg(x, tab);
            const dflt ir3 = df_mul(ir, ir2), ir5 = df_mul(ir3, ir2);
            const dflt b1 = df_mul(df_sub(ONE, e), ir3);
            const dflt b2 = df_mul(df_mul(THREE, df_sub(ONE, df_mul(df_add(ONE, x), e))), ir5);
            const dflt vx = {vh.x, vl.x}, vy = {vh.y, vl.y}, vz = {vh.z, vl.z};
            const dflt s = df_mul(b2, df_madd(R[2], vz, df_madd(R[1], vy, df_mul(R[0], vx))));
            sx = df_add(sx, df_sub(df_mul(s, R[0]), df_mul(b1, vx)));
            sy = df_add(sy, df_sub(df_mul(s, R[1]), df_mul(b1, vy)));
            sz = df_add(sz, df_sub(df_mul(s, R[2]), df_mul(b1, vz)));
          }
      }
    } else {
      const float4 pi = A.p32[gi];
      const float2 mi = A.tm32[gi];
      const bool perm = act == A_E0;
      for (int j0 = 0; j0 < info.n; j0 += kChunk) {
        __syncthreads();
        const int jl = j0 + threadIdx.x;
        if (jl < info.n) {
          const long long g = info.off + jl;
          st.a[threadIdx.x] = A.p32[g];
          const float2 m = A.tm32[g];
          st.e[threadIdx.x] = make_float4(m.x, m.y, 0.f, 0.f);
          if (perm) {
            st.b[threadIdx.x] = A.mp32[3 * g];
            st.c[threadIdx.x] = A.mp32[3 * g + 1];
            st.d[threadIdx.x] = A.mp32[3 * g + 2];
          } else {
            st.b[threadIdx.x] = A.v32[g];
          }
        }
        __syncthreads();
        const int cnt = min(kChunk, info.n - j0);
        float fx = 0.f, fy = 0.f, fz = 0.f;
        if (valid)
          for (int k = h; k < cnt; k += 2) {
            if (j0 + k == il) continue;
            const float4 pj = st.a[k];
            const float4 tj = st.e[k];
            if (perm && __float_as_int(tj.y) == __float_as_int(mi.y)) continue;  // same molecule: excluded
            const float rx = pi.x - pj.x, ry = pi.y - pj.y, rz = pi.z - pj.z;
            const float r2 = rx * rx + ry * ry + rz * rz;
            float b1, b2, b3;
            thole32(r2, fminf(mi.x, tj.x), pi.w * pj.w, b1, b2, b3, perm);
            if (perm) {
              const float4 m0 = st.b[k], m1 = st.c[k], m2 = st.d[k];
              // q, d, Theta (xx, yy, zz, xy, xz, yz) of j
              const float tx = m1.x * rx + m1.w * ry + m2.x * rz;
              const float ty = m1.w * rx + m1.y * ry + m2.y * rz;
              const float tz = m2.x * rx + m2.y * ry + m1.z * rz;
              const float rtr = rx * tx + ry * ty + rz * tz;
              const float dr = m0.y * rx + m0.z * ry + m0.w * rz;
              const float rad = m0.x * b1 + b2 * dr + b3 * rtr * (1.f / 3.f);
              const float c2 = b2 * (2.f / 3.f);
              fx += rad * rx - b1 * m0.y - c2 * tx;
              fy += rad * ry - b1 * m0.z - c2 * ty;
              fz += rad * rz - b1 * m0.w - c2 * tz;
            } else {
              const float4 v = st.b[k];
              const float s = b2 * (v.x * rx + v.y * ry + v.z * rz);
              fx += s * rx - b1 * v.x;
              fy += s * ry - b1 * v.y;
              fz += s * rz - b1 * v.z;
            }
          }
        acc_add(sx, fx);
        acc_add(sy, fy);
        acc_add(sz, fz);
      }
    }
    // the two threads of a row add their sums (same order in both)
    {
      dflt o;
      o.hi = __shfl_xor_sync(0xffffffffu, sx.hi, 1);
      o.lo = __shfl_xor_sync(0xffffffffu, sx.lo, 1);
      sx = h == 0 ? df_add(sx, o) : df_add(o, sx);
      o.hi = __shfl_xor_sync(0xffffffffu, sy.hi, 1);
      o.lo = __shfl_xor_sync(0xffffffffu, sy.lo, 1);
      sy = h == 0 ? df_add(sy, o) : df_add(o, sy);
      o.hi = __shfl_xor_sync(0xffffffffu, sz.hi, 1);
      o.lo = __shfl_xor_sync(0xffffffffu, sz.lo, 1);
      sz = h == 0 ? df_add(sz, o) : df_add(o, sz);
    }
    // ---- epilogue in float64
    double rz = 0.0, zw = 0.0;
    if (valid && h == 0) {
      const double4_32a t = make_double4_32a(df_to_double(sx), df_to_double(sy), df_to_double(sz), 0.0);
      if (act == A_E0) {
        A.e0[gi] = t;
      } else if (act == A_TVI) {
        const double ia = A.al[gi].y;
        const double4_32a z = A.z[gi], r = A.r[gi];
        const double4_32a wv = make_double4_32a(z.x * ia - t.x, z.y * ia - t.y, z.z * ia - t.z, 0.0);
        A.w[gi] = wv;
        rz = r.x * z.x + r.y * z.y + r.z * z.z;
        zw = z.x * wv.x + z.y * wv.y + z.z * wv.z;
      } else {
        A.tmp[gi] = t;  // A_TV (initial residual) and A_CHECK
      }
    }
    if (act == A_TVI) {
      const double a = block_sum(rz, red), b = block_sum(zw, red);
      if (threadIdx.x == 0) {
        A.part_rz[info.tile0 + tile] = a;
        A.part_zw[info.tile0 + tile] = b;
      }
    }
  }
}

__global__ void __launch_bounds__(kThreads) k_batch_vectors(Arena A, int n_items, const int2* __restrict__ items,
                                                            int* __restrict__ heads) {
  __shared__ double red[kThreads / 32];
  __shared__ double bc;
  __shared__ double sbeta, sgamma;
  __shared__ bool sbad;
  if (blockIdx.x == 0 && threadIdx.x == 0) heads[0] = 0;  // the pair phase's queue, for the next launch
  while (true) {
    const int it = next_item(heads + 1);
    if (it >= n_items) break;
    const int2 w = items[it];
    const int rq = w.x, tile = w.y;
    const ReqInfo info = A.info[rq];
    // what the pair phase of the launch before did for this request; only
    // tile 0 reads and rewrites the request's ReqT in this launch
    const ReqS s = A.reqS[rq];
    const int act = s.act;
    if (act == A_IDLE) continue;
    const int i0 = tile * kRows;
    const int nloc = min(kRows, info.n - i0);
    if (act == A_FINISH) {
      if (tile == 0 && threadIdx.x == 0) A.reqT[rq].kind = K_DONE;
      continue;
    }
    double beta = 0.0, gamma = 0.0;
    if (act == A_TVI) {
      const double rho = reduce_tiles(A.part_rz, info.tile0, info.ntiles, &bc);
      const double m = reduce_tiles(A.part_zw, info.tile0, info.ntiles, &bc);
      if (threadIdx.x == 0) {
        double b = 0.0, den = m;
        if (!s.first) {
          b = rho / s.rho_old;
          den = m - b * rho / s.gamma_old;
        }
        sbad = !(den > 0.0);  // p.Ap <= 0: not positive definite
        sbeta = b;
        sgamma = rho / den;
        if (tile == 0) {
          ReqT nt = A.reqT[rq];
          if (sbad) {
            nt.kind = K_DONE;
            ReqOut o;
            o.status = 3;
            o.iters = s.iter + 1;
            o.rms = s.rms;
            o.U = 0.0;
            A.out[rq] = o;
          } else {
            nt.kind = K_ITER;
            nt.iter = s.iter + 1;
            nt.first = 0;
            nt.rho = rho;
            nt.gamma = rho / den;
          }
          A.reqT[rq] = nt;
        }
      }
      __syncthreads();
      if (sbad) continue;
      beta = sbeta;
      gamma = sgamma;
    } else if (tile == 0 && threadIdx.x == 0) {
      ReqT nt = A.reqT[rq];
      if (act == A_E0) {
        nt.kind = K_INIT;
      } else {  // A_TV (initial residual) or A_CHECK: restart from the residual
        nt.kind = act == A_TV ? K_ITER : K_AFTER;
        nt.first = 1;
      }
      A.reqT[rq] = nt;
    }
    double zz = 0.0, me = 0.0;
    const int k = threadIdx.x;
    if (k < nloc) {
      const long long g = info.off + i0 + k;
      const double2 al = A.al[g];
      const double4_32a e0 = A.e0[g];
      if (act == A_E0) {
        const double4_32a mu = make_double4_32a(al.x * e0.x, al.x * e0.y, al.x * e0.z, 0.0);
        A.mu[g] = mu;
        A.v32[g] = make_float4(__double2float_rn(mu.x), __double2float_rn(mu.y), __double2float_rn(mu.z), 0.f);
      } else {
        double4_32a mu = A.mu[g], r, z;
        if (act == A_TVI) {
          const double4_32a zv = A.z[g], wv = A.w[g];
          double4_32a p = A.p[g], q = A.q[g];
          r = A.r[g];
          p = make_double4_32a(zv.x + beta * p.x, zv.y + beta * p.y, zv.z + beta * p.z, 0.0);
          q = make_double4_32a(wv.x + beta * q.x, wv.y + beta * q.y, wv.z + beta * q.z, 0.0);
          mu = make_double4_32a(mu.x + gamma * p.x, mu.y + gamma * p.y, mu.z + gamma * p.z, 0.0);
          r = make_double4_32a(r.x - gamma * q.x, r.y - gamma * q.y, r.z - gamma * q.z, 0.0);
          A.p[g] = p;
          A.q[g] = q;
          A.mu[g] = mu;
        } else {  // r = E0 - mu/alpha + T mu
          const double4_32a t = A.tmp[g];
          r = make_double4_32a(e0.x - mu.x * al.y + t.x, e0.y - mu.y * al.y + t.y, e0.z - mu.z * al.y + t.z, 0.0);
        }
        z = make_double4_32a(al.x * r.x, al.x * r.y, al.x * r.z, 0.0);
        A.r[g] = r;
        A.z[g] = z;
        A.v32[g] = make_float4(__double2float_rn(z.x), __double2float_rn(z.y), __double2float_rn(z.z), 0.f);
        zz = z.x * z.x + z.y * z.y + z.z * z.z;
        me = mu.x * e0.x + mu.y * e0.y + mu.z * e0.z;
      }
    }
    if (act != A_E0) {
      const double a = block_sum(zz, red), b = block_sum(me, red);
      if (threadIdx.x == 0) {
        A.partz[info.tile0 + tile] = a;
        A.parte[info.tile0 + tile] = b;
      }
    }
  }
}

// Per-atom records of an admitted request from its float64 inputs (device,
// caller order, written into the arena range by the host's copies): the
// float32 records of the pair phase, the double-float records of the check,
// (alpha, 1/alpha).
__global__ void k_batch_records(int off, int n, const double* __restrict__ xyz, const double* __restrict__ q,
                                const double* __restrict__ dip, const double* __restrict__ quad,
                                const double* __restrict__ alpha, const double* __restrict__ thole,
                                const int* __restrict__ mol, Arena A, int* __restrict__ bad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const long long g = off + i;
  const double al = alpha[i];
  if (!(al > 0.0)) atomicOr(bad, 1);
  const double isa = al > 0.0 ? 1.0 / sqrt(al) : 0.0;
  const double x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
  A.p32[g] = make_float4((float)x, (float)y, (float)z, (float)isa);
  A.tm32[g] = make_float2((float)thole[i], __int_as_float(mol[i]));
  const double* Q = quad + 6 * i;
  A.mp32[3 * g] = make_float4((float)q[i], (float)dip[3 * i], (float)dip[3 * i + 1], (float)dip[3 * i + 2]);
  A.mp32[3 * g + 1] = make_float4((float)Q[0], (float)Q[1], (float)Q[2], (float)Q[3]);
  A.mp32[3 * g + 2] = make_float4((float)Q[4], (float)Q[5], 0.f, 0.f);
  const dflt sx = df_split(x), sy = df_split(y), sz = df_split(z), si = df_split(isa), st = df_split(thole[i]);
  A.pdf[3 * g] = make_float4(sx.hi, sy.hi, sz.hi, si.hi);
  A.pdf[3 * g + 1] = make_float4(sx.lo, sy.lo, sz.lo, si.lo);
  A.pdf[3 * g + 2] = make_float4(st.hi, st.lo, __int_as_float(mol[i]), 0.f);
  A.al[g] = make_double2(al, al > 0.0 ? 1.0 / al : 0.0);
  const double4_32a zero = make_double4_32a(0.0, 0.0, 0.0, 0.0);
  A.p[g] = zero;
  A.q[g] = zero;
}

// The converged dipoles of a request in caller order [n][3].
__global__ void k_batch_result(int off, int n, const double4_32a* __restrict__ mu, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double4_32a m = mu[off + i];
  out[3 * i] = m.x;
  out[3 * i + 1] = m.y;
  out[3 * i + 2] = m.z;
}

}  // namespace batch
}  // namespace amp
