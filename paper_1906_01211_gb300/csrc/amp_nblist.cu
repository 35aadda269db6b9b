// Cell list and neighbour lists (kernel a).
//
// The paper's list builder is cell based (Section "Hotspots": mlistcell) and
// its selection loops build a mask of the neighbours inside the cutoff and then
// pack their indices (Section "Typical selection loop"). On the GPU the mask is
// a warp ballot and the packing is a popcount prefix, which also keeps the
// packed order deterministic (lane order). Rows are scanned in cell order, so
// the atoms of a cell are contiguous (the "sorting indexes" the paper's
// conclusion proposes for faster indexing).
//
// Steps:
//   1. cell of every atom (wrapped position), counts per cell;
//   2. exclusive scan -> cell_start; scatter; stable sort inside each cell by
//      the caller's index, so the cell order does not depend on atomics;
//   3. gather the atom records into cell order (float64 + wrapped float32);
//   4. one warp per atom scans the candidates in the cells within two cells
//      per axis (cell edge >= rc/2), as runs of consecutive atoms along z,
//      each run trimmed to the cells within reach of the atom and all runs
//      packed 32 candidates to a round: float32 distance pre-filter with a
//      margin, exact float64 decision d.d < rc^2 for candidates near the
//      cutoff; counts, and the owned neighbours into a slab row;
//   5. scan the row counts; copy the slab rows into the full rows and the half
//      list (or, if a slab row overflowed, scan the candidates again and write
//      them at the row offsets);
//   6. each pair id is scattered to its non-owner's row, which sorts that part
//      of the row by pair id (deterministic order).
#include <cmath>
#include <cstring>
#include <cstdarg>
#include <cstdio>

#include "amp_internal.cuh"

namespace amp {

int fail(amp_ctx* c, int code, const char* fmt, ...) {
  if (c) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(c->err, sizeof(c->err), fmt, ap);
    va_end(ap);
  }
  return code;
}

int cuda_check(amp_ctx* c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return AMP_OK;
  return fail(c, AMP_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

namespace {

__device__ __forceinline__ double wrap_box(double x, double L) {
  double w = x - L * floor(x / L);
  if (w >= L) w -= L;
  if (w < 0.0) w += L;
  if (w >= L) w = 0.0;
  return w;
}

__global__ void k_cell_assign(int n, const double* __restrict__ xyz, double L, int nc,
                              int* __restrict__ cell_of, int* __restrict__ cell_count) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int c[3];
  for (int a = 0; a < 3; ++a) {
    double w = wrap_box(xyz[3 * i + a], L);
    int k = (int)(w * (double)nc / L);
    c[a] = k < 0 ? 0 : (k >= nc ? nc - 1 : k);
  }
  int id = (c[0] * nc + c[1]) * nc + c[2];
  cell_of[i] = id;
  atomicAdd(&cell_count[id], 1);
}

// Single-block exclusive scan: out[k] = sum_{m<k} in[k], out[n] = total. A
// second block, if launched, scans (in2, out2) the same way.
__global__ void k_scan_exclusive(const int* __restrict__ in, int* __restrict__ out, int n,
                                 const int* __restrict__ in2 = nullptr, int* __restrict__ out2 = nullptr) {
  if (blockIdx.x == 1) {
    in = in2;
    out = out2;
  }
  __shared__ int warp_sums[32];
  __shared__ int carry;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int per = (n + blockDim.x - 1) / blockDim.x;
  const int lo = min(n, t * per), hi = min(n, lo + per);
  int s = 0;
  for (int k = lo; k < hi; ++k) s += in[k];
  int v = s;
  for (int o = 1; o < 32; o <<= 1) {
    int u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  if (lane == 31) warp_sums[w] = v;
  __syncthreads();
  if (w == 0) {
    int nw = blockDim.x >> 5;
    int x = lane < nw ? warp_sums[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      int u = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += u;
    }
    if (lane < nw) warp_sums[lane] = x;
    if (lane == nw - 1) carry = x;
  }
  __syncthreads();
  int run = v - s + (w > 0 ? warp_sums[w - 1] : 0);
  for (int k = lo; k < hi; ++k) {
    out[k] = run;
    run += in[k];
  }
  if (t == 0) out[n] = carry;
}

__global__ void k_cell_scatter(int n, const int* __restrict__ cell_of, const int* __restrict__ cell_start,
                               int* __restrict__ cell_fill, int* __restrict__ slot_tmp) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int c = cell_of[i];
  int slot = cell_start[c] + atomicAdd(&cell_fill[c], 1);
  slot_tmp[slot] = i;
}

// One warp per cell: rank of each member by caller index -> stable order.
__global__ void k_cell_sort(int ncell, const int* __restrict__ cell_start, const int* __restrict__ slot_tmp,
                            int* __restrict__ perm) {
  int cell = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (cell >= ncell) return;
  int s = cell_start[cell], e = cell_start[cell + 1];
  for (int k = s + lane; k < e; k += 32) {
    int me = slot_tmp[k];
    int rank = 0;
    for (int m = s; m < e; ++m) rank += slot_tmp[m] < me;
    perm[s + rank] = me;
  }
}

__global__ void k_gather_atoms(int n, const int* __restrict__ perm, const double* __restrict__ xyz,
                               const double* __restrict__ q, const double* __restrict__ dip,
                               const double* __restrict__ quad, const double* __restrict__ alpha,
                               const double* __restrict__ thole, const int* __restrict__ mol, double L,
                               int* __restrict__ inv_perm, double4_32a* __restrict__ A, double4_32a* __restrict__ B,
                               double4_32a* __restrict__ C, double4_32a* __restrict__ D, float4* __restrict__ pos32,
                               const int* __restrict__ cell_of, int* __restrict__ cell_sorted,
                               double2* __restrict__ alph, int* __restrict__ flags) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  int i = perm[s];
  inv_perm[i] = s;
  cell_sorted[s] = cell_of[i];
  double x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
  double al = alpha[i];
  if (!(al > 0.0)) atomicOr(&flags[0], 2);
  alph[s] = make_double2(al, 1.0 / al);
  A[s] = make_double4_32a(x, y, z, q[i]);
  B[s] = make_double4_32a(dip[3 * i], dip[3 * i + 1], dip[3 * i + 2], 1.0 / sqrt(al));
  C[s] = make_double4_32a(quad[6 * i], quad[6 * i + 1], quad[6 * i + 2], quad[6 * i + 3]);
  D[s] = make_double4_32a(quad[6 * i + 4], quad[6 * i + 5], thole[i], (double)mol[i]);
  pos32[s] = make_float4((float)wrap_box(x, L), (float)wrap_box(y, L), (float)wrap_box(z, L), 0.f);
}

struct ListParams {
  int n, nc;  // atoms, cells per axis (edge >= rc / 2)
  int slab;   // slab row capacity (kMode 2)
  double L, rc2;
  float Lf, invLf, lo2, hi2;
  float hcell;   // cell edge L / nc
  float reach2;  // (rc + 0.05)^2: a cell farther than this from the atom holds no candidate
};

// Exact float64 decision, operation by operation as the plain definition
// d = x_i - x_j; d -= L * rint(d / L); d.d < rc^2 (no contraction).
__device__ __forceinline__ bool exact_in_range(const double4_32a& a, const double4_32a& b, double L, double rc2) {
  double dx = __dsub_rn(a.x, b.x), dy = __dsub_rn(a.y, b.y), dz = __dsub_rn(a.z, b.z);
  dx = __dsub_rn(dx, __dmul_rn(L, rint(dx / L)));
  dy = __dsub_rn(dy, __dmul_rn(L, rint(dy / L)));
  dz = __dsub_rn(dz, __dmul_rn(L, rint(dz / L)));
  double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
  return r2 < rc2;
}

// One round of 32 candidates of row i (lane: candidate k, in range or not):
// owned pairs (rule (i < k) != (i + k odd)) open the row, the full slot and
// the pair id sharing the rank. kMode 0 counts; 1 writes at the row offsets;
// 2 writes the owned neighbours into the slab row srow (capacity slab_cap).
template <int kMode>
__device__ __forceinline__ void emit_round(bool in, int i, int k, unsigned lt, int& nfull, int& nhalf, int fbase,
                                           int hbase, int* srow, int slab_cap, int* __restrict__ full_j,
                                           int* __restrict__ full_ref, int* __restrict__ half_i,
                                           int* __restrict__ half_j) {
  const bool own = in && ((i < k) != (((i + k) & 1) != 0));
  const unsigned mf = __ballot_sync(0xffffffffu, in);
  const unsigned mh = __ballot_sync(0xffffffffu, own);
  if (own) {
    const int rank = nhalf + __popc(mh & lt);
    if (kMode == 1) {
      const int pid = hbase + rank;
      full_j[fbase + rank] = k;
      full_ref[fbase + rank] = pid << 1;
      half_i[pid] = i;
      half_j[pid] = k;
    } else if (kMode == 2 && rank < slab_cap) {
      srow[rank] = k;
    }
  }
  nfull += __popc(mf);
  nhalf += __popc(mh);
}

// Candidates of atom i: cells within two cells per axis (cell edge >= rc/2;
// every cell when there are fewer than five per axis). For each (x, y) cell
// column the z cells form one or two runs of consecutive cells, hence of
// consecutive atoms; the runs of all columns are scanned 32 candidates at a
// time, in a fixed order (so the rows come out in the same order whatever
// the trimming of the runs). kMode 0 counts the full and owned
// neighbours; 1 writes them at the row offsets; 2 counts and writes the owned
// neighbours into a slab row of P.slab entries (flag bit 4 if one overflows),
// so that a single scan of the candidates suffices.
template <int kMode>
__global__ void k_neighbours(ListParams P, const float4* __restrict__ pos32, const double4_32a* __restrict__ A,
                             const int* __restrict__ cell_sorted, const int* __restrict__ cell_start,
                             int* __restrict__ full_cnt, int* __restrict__ half_cnt,
                             const int* __restrict__ full_start, const int* __restrict__ half_start,
                             int* __restrict__ full_j, int* __restrict__ full_ref, int* __restrict__ half_i,
                             int* __restrict__ half_j, int* __restrict__ slab, int* __restrict__ flags) {
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= P.n) return;
  const unsigned lt = (1u << lane) - 1u;
  const float4 pi = pos32[i];
  const double4_32a ai = A[i];
  const int nc = P.nc;
  const int cself = cell_sorted[i];  // the cell the atom was binned in (float64 wrap)
  const int ci[3] = {cself / (nc * nc), (cself / nc) % nc, cself % nc};
  const bool all = nc < 5;
  const int span = all ? nc : 5;
  int nfull = 0, nhalf = 0;
  const int fbase = kMode == 1 ? full_start[i] : 0;
  const int hbase = kMode == 1 ? half_start[i] : 0;
  int* srow = kMode == 2 ? slab + (long long)i * P.slab : nullptr;
  // Lane c < span^2 holds column c's z runs up front: run 0 the cells
  // without a periodic shift, run 1 the wrapped ones. With five or more cells
  // per axis the image of a candidate follows from its cell offset: the run's
  // atoms are compared with atom i moved by minus that image shift (sx, sy per
  // column, sz for run 1), which is the minimum image of every candidate
  // within the cutoff; the runs are trimmed to the cells whose nearest point
  // lies within the list radius (plus a margin far above the rounding of the
  // float positions), so a trimmed cell holds no candidate that could be
  // emitted. With fewer cells the float minimum image is taken per candidate
  // and nothing is trimmed.
  const int ncol = span * span;
  int st0 = 0, len0 = 0, st1 = 0, len1 = 0, code = 0;  // code: x and y shift + 1, two bits each
  if (lane < ncol) {
    const int ox = lane / span, oy = lane % span;
    if (all) {
      const int base = (ox * nc + oy) * nc;
      st0 = cell_start[base];
      len0 = cell_start[base + nc] - st0;
      code = 1 | (1 << 2);
    } else {
      const int cxr = ci[0] + ox - 2, cyr = ci[1] + oy - 2;  // unwrapped
      const int cx = (cxr + nc) % nc, cy = (cyr + nc) % nc;
      code = (cxr < 0 ? 0 : (cxr >= nc ? 2 : 1)) | ((cyr < 0 ? 0 : (cyr >= nc ? 2 : 1)) << 2);
      const float h = P.hcell;
      const float dxm = fmaxf(0.f, fmaxf((float)cxr * h - pi.x, pi.x - (float)(cxr + 1) * h));
      const float dym = fmaxf(0.f, fmaxf((float)cyr * h - pi.y, pi.y - (float)(cyr + 1) * h));
      const float rem = P.reach2 - (dxm * dxm + dym * dym);
      if (rem >= 0.f) {
        int zlo = ci[2] - 2, zhi = ci[2] + 2;  // unwrapped z cells kept: [zlo, zhi]
        for (; zlo < ci[2]; ++zlo) {
          const float d = pi.z - (float)(zlo + 1) * h;
          if (d * d <= rem) break;
        }
        for (; zhi > ci[2]; --zhi) {
          const float d = (float)zhi * h - pi.z;
          if (d * d <= rem) break;
        }
        const int base = (cx * nc + cy) * nc;
        const int a = max(zlo, 0), b = min(zhi, nc - 1);
        if (a <= b) {
          st0 = cell_start[base + a];
          len0 = cell_start[base + b + 1] - st0;
        }
        if (zlo < 0) {
          st1 = cell_start[base + zlo + nc];
          len1 = cell_start[base + nc] - st1;
        } else if (zhi >= nc) {
          st1 = cell_start[base];
          len1 = cell_start[base + zhi - nc + 1] - st1;
        }
      }
    }
  }
  // The candidates of all runs, in column order and run 0 before run 1,
  // packed 32 to a round: lane t of a round finds its column by a binary
  // search over the inclusive prefix sums of the column lengths.
  const int tot = len0 + len1;
  int inc = tot;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int u = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += u;
  }
  const int total = __shfl_sync(0xffffffffu, inc, 31);
  const int exc = inc - tot;
  const float sz1 = all ? 0.f : (ci[2] - 2 < 0 ? -P.Lf : P.Lf);  // shift of every run 1
  for (int t0 = 0; t0 < total; t0 += 32) {
    const int t = t0 + lane;
    int col = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
      const int v = __shfl_sync(0xffffffffu, inc, col + step - 1);
      if (v <= t) col += step;
    }
    const int ex = __shfl_sync(0xffffffffu, exc, col), l0 = __shfl_sync(0xffffffffu, len0, col);
    const int s0 = __shfl_sync(0xffffffffu, st0, col), s1 = __shfl_sync(0xffffffffu, st1, col);
    const int cd = __shfl_sync(0xffffffffu, code, col);
    bool in = false;
    int k = -1;
    if (t < total) {
      const int o = t - ex;
      const float sx = (float)((cd & 3) - 1) * P.Lf, sy = (float)((cd >> 2) - 1) * P.Lf;
      float sz = 0.f;
      if (o < l0) {
        k = s0 + o;
      } else {
        k = s1 + (o - l0);
        sz = sz1;
      }
      if (k != i) {
        const float4 pj = pos32[k];
        const float px = pi.x - sx, py = pi.y - sy, pz = pi.z - sz;
        float dx = pj.x - px, dy = pj.y - py, dz = pj.z - pz;
        if (all) {
          dx -= P.Lf * rintf(dx * P.invLf);
          dy -= P.Lf * rintf(dy * P.invLf);
          dz -= P.Lf * rintf(dz * P.invLf);
        }
        const float r2 = dx * dx + dy * dy + dz * dz;
        if (r2 < P.hi2) in = (r2 <= P.lo2) ? true : exact_in_range(ai, A[k], P.L, P.rc2);
      }
    }
    emit_round<kMode>(in, i, k, lt, nfull, nhalf, fbase, hbase, srow, P.slab, full_j, full_ref, half_i, half_j);
  }
  if (kMode != 1 && lane == 0) {
    full_cnt[i] = nfull;
    half_cnt[i] = nhalf;
    if (kMode == 2 && nhalf > P.slab) atomicOr(flags, 4);
  }
}

// The same list from stored candidates: row i of (cand_start, cand_j) holds
// the pairs that were within cutoff + skin at the last cell search; the
// in-range decision (float prefilter, float64 operations near the cutoff) and
// the emission are those of k_neighbours, with the float minimum image per
// candidate (the atoms have moved since the candidates were found).
template <int kMode>
__global__ void k_filter(ListParams P, const float4* __restrict__ pos32, const double4_32a* __restrict__ A,
                         const int* __restrict__ cand_start, const int* __restrict__ cand_j,
                         int* __restrict__ full_cnt, int* __restrict__ half_cnt,
                         const int* __restrict__ full_start, const int* __restrict__ half_start,
                         int* __restrict__ full_j, int* __restrict__ full_ref, int* __restrict__ half_i,
                         int* __restrict__ half_j, int* __restrict__ slab, int* __restrict__ flags) {
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= P.n) return;
  const unsigned lt = (1u << lane) - 1u;
  const float4 pi = pos32[i];
  const double4_32a ai = A[i];
  int nfull = 0, nhalf = 0;
  const int fbase = kMode == 1 ? full_start[i] : 0;
  const int hbase = kMode == 1 ? half_start[i] : 0;
  int* srow = kMode == 2 ? slab + (long long)i * P.slab : nullptr;
  const int s = cand_start[i], e = cand_start[i + 1];
  for (int k0 = s; k0 < e; k0 += 32) {
    const int kk = k0 + lane;
    int k = 0;
    bool in = false;
    if (kk < e) {
      k = cand_j[kk];
      const float4 pj = pos32[k];
      float dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
      dx -= P.Lf * rintf(dx * P.invLf);
      dy -= P.Lf * rintf(dy * P.invLf);
      dz -= P.Lf * rintf(dz * P.invLf);
      const float r2 = dx * dx + dy * dy + dz * dz;
      if (r2 < P.hi2) in = (r2 <= P.lo2) ? true : exact_in_range(ai, A[k], P.L, P.rc2);
    }
    emit_round<kMode>(in, i, k, lt, nfull, nhalf, fbase, hbase, srow, P.slab, full_j, full_ref, half_i, half_j);
  }
  if (kMode != 1 && lane == 0) {
    full_cnt[i] = nfull;
    half_cnt[i] = nhalf;
    if (kMode == 2 && nhalf > P.slab) atomicOr(flags, 4);
  }
}

// Largest squared minimum-image displacement of the caller's new positions
// xyz [N][3] from the sorted reference positions ref, as float bits (non-
// negative floats order like their bits) in *dmax (zeroed by the caller).
__global__ void __launch_bounds__(256) k_displacement(int n, const int* __restrict__ perm,
                                                      const double* __restrict__ xyz,
                                                      const double4_32a* __restrict__ ref, double L,
                                                      int* __restrict__ dmax) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  float d2 = 0.f;
  if (s < n) {
    const int i = perm[s];
    const double4_32a r = ref[s];
    double dx = xyz[3 * i] - r.x, dy = xyz[3 * i + 1] - r.y, dz = xyz[3 * i + 2] - r.z;
    dx -= L * rint(dx / L);
    dy -= L * rint(dy / L);
    dz -= L * rint(dz / L);
    d2 = (float)(dx * dx + dy * dy + dz * dz);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) d2 = fmaxf(d2, __shfl_xor_sync(0xffffffffu, d2, o));
  if ((threadIdx.x & 31) == 0) atomicMax(dmax, __float_as_int(d2));
}

// New positions into the sorted per-atom records (A.xyz, float copies), the
// other inputs unchanged.
__global__ void k_apply_positions(int n, const int* __restrict__ perm, const double* __restrict__ xyz, double L,
                                  double4_32a* __restrict__ A, float4* __restrict__ pos32) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int i = perm[s];
  const double x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
  double4_32a a = A[s];
  a.x = x;
  a.y = y;
  a.z = z;
  A[s] = a;
  pos32[s] = make_float4((float)wrap_box(x, L), (float)wrap_box(y, L), (float)wrap_box(z, L), 0.f);
}

// Speculative fill (the lists were sized by an earlier call): the fill kernels
// run before the host has read the new counts and do nothing when a slab row
// overflowed (flag bit 4) or the lists do not fit their buffers (then they set
// flag bit 8); the host checks both after its single synchronisation and
// refills on the two-pass path.
struct ListGuard {
  const int* flags;  // null: counts known on the host, nothing to check
  int n;
  long long cap_full, cap_half;
};

__device__ __forceinline__ bool list_skip(const ListGuard& g, const int* full_start, const int* half_start,
                                          int* flags) {
  if (!g.flags) return false;
  if (*g.flags & 4) return true;
  if (full_start[g.n] > g.cap_full || half_start[g.n] > g.cap_half) {
    atomicOr(flags, 8);
    return true;
  }
  return false;
}

// Slab rows -> owned part of the full rows and the half list.
__global__ void k_slab_copy(int n, int slab_cap, const int* __restrict__ slab, const int* __restrict__ half_cnt,
                            const int* __restrict__ full_start, const int* __restrict__ half_start,
                            int* __restrict__ full_j, int* __restrict__ full_ref, int* __restrict__ half_i,
                            int* __restrict__ half_j, ListGuard g, int* __restrict__ flags) {
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= n || list_skip(g, full_start, half_start, flags)) return;
  const int m = half_cnt[i], fb = full_start[i], hb = half_start[i];
  const int* row = slab + (long long)i * slab_cap;
  for (int r = lane; r < m; r += 32) {
    const int k = row[r], pid = hb + r;
    full_j[fb + r] = k;
    full_ref[fb + r] = pid << 1;
    half_i[pid] = i;
    half_j[pid] = k;
  }
}

// The rest of row j lists the pairs owned by other rows: every pair id is
// scattered to its non-owner's row (atomic slot), then each row sorts that part
// by pair id, so the final order does not depend on the atomics.
__global__ void k_transpose_scatter(long long nh, const int* __restrict__ half_j,
                                    const int* __restrict__ full_start, const int* __restrict__ half_cnt,
                                    int* __restrict__ tcount, int* __restrict__ tmp, ListGuard g,
                                    const int* __restrict__ half_start, int* __restrict__ flags) {
  const long long pid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g.flags) nh = half_start[g.n];  // speculative: the count is on the device only
  if (pid >= nh || list_skip(g, full_start, half_start, flags)) return;
  const int j = half_j[pid];
  const int slot = full_start[j] + half_cnt[j] + atomicAdd(&tcount[j], 1);
  tmp[slot] = (int)pid;
}

constexpr int kSortCap = 256;  // transposed entries per row staged in shared memory

__global__ void __launch_bounds__(256) k_transpose_sort(int n, const int* __restrict__ full_start,
                                                        const int* __restrict__ half_cnt,
                                                        const int* __restrict__ tmp, const int* __restrict__ half_i,
                                                        int* __restrict__ full_j, int* __restrict__ full_ref,
                                                        int* __restrict__ pos_tr, ListGuard g,
                                                        const int* __restrict__ half_start, int* __restrict__ flags) {
  __shared__ int stage[256 / 32][kSortCap];
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (i >= n || list_skip(g, full_start, half_start, flags)) return;  // whole warps leave together
  const int lo = full_start[i] + half_cnt[i], hi = full_start[i + 1], m = hi - lo;
  const bool staged = m <= kSortCap;
  if (staged)
    for (int e = lane; e < m; e += 32) stage[w][e] = tmp[lo + e];
  __syncwarp();
  for (int e = lane; e < m; e += 32) {
    const int p = staged ? stage[w][e] : tmp[lo + e];
    int rank = 0;
    if (staged)
      for (int q = 0; q < m; ++q) rank += stage[w][q] < p;
    else
      for (int q = lo; q < hi; ++q) rank += tmp[q] < p;
    full_ref[lo + rank] = (p << 1) | 1;
    full_j[lo + rank] = half_i[p];
    pos_tr[p] = lo + rank;
  }
}

// The list totals and the build flags into the mapped host readback
// (hibuf[0], hibuf[1], hibuf[2, 6)), after every kernel that sets a flag.
__global__ void k_list_readback(const int* __restrict__ full_total, const int* __restrict__ half_total,
                                const int* __restrict__ flags, int* __restrict__ h) {
  if (threadIdx.x == 0) {
    h[0] = *full_total;
    h[1] = *half_total;
    for (int k = 0; k < 4; ++k) h[2 + k] = flags[k];
  }
}

}  // namespace

namespace {

// Slab rows for the single-pass list: four times the mean number of owned
// neighbours (half of 4/3 pi rc^3 n / L^3) within rc, at least 64; a row that
// would overflow sends the build through the two-pass count / fill path.
int list_params(amp_ctx* c, double rc, ListParams* P) {
  const int n = c->n;
  const double L = c->cfg.box;
  const double mean_full = 4.0 / 3.0 * M_PI * rc * rc * rc * (double)n / (L * L * L);
  int slab = (int)std::ceil(2.0 * mean_full / 32.0) * 32;
  if (slab < 64) slab = 64;
  if (slab > 4096) slab = 4096;
  if ((long long)n * slab > c->slab_cap) {
    dev_free(c, c->slab);
    c->slab = nullptr;
    c->slab_cap = 0;
    int r;
    if ((r = dev_alloc(c, &c->slab, (long long)n * slab))) return r;
    c->slab_cap = (long long)n * slab;
  }
  P->n = n;
  P->nc = c->nc;
  P->slab = slab;
  P->L = L;
  P->rc2 = rc * rc;
  P->Lf = (float)L;
  P->invLf = (float)(1.0 / L);
  P->lo2 = (float)(rc * rc - 0.01);
  P->hi2 = (float)(rc * rc + 0.01);
  P->hcell = (float)(L / (double)(c->nc > 0 ? c->nc : 1));
  P->reach2 = (float)((rc + 0.05) * (rc + 0.05));
  return AMP_OK;
}

// After the counting (and slab) pass of the cell search or of the candidate
// filter: row offsets, the fill, one host round trip. Lists sized by an
// earlier call are filled before the counts reach the host; the fill kernels
// skip themselves if the lists outgrew the buffers or a slab row overflowed,
// and the two-pass path below redoes the fill (second pass of the same source).
int finish_lists(amp_ctx* c, const ListParams& P, bool from_candidates) {
  const int n = c->n, slab = P.slab;
  cudaStream_t st = c->stream;
  const int lb = amp_blocks((long long)n * 32, 256);
  int r;
  k_scan_exclusive<<<2, 1024, 0, st>>>(c->full_cnt, c->full_start, n, c->half_cnt, c->half_start);
  if ((r = cuda_check(c, cudaGetLastError(), "list count launch"))) return r;
  const bool speculative = c->cap_full > 0 && c->cap_half > 0;
  const ListGuard none{nullptr, n, 0, 0};
  if (speculative) {
    const ListGuard g{c->flags, n, c->cap_full, c->cap_half};
    k_slab_copy<<<lb, 256, 0, st>>>(n, slab, c->slab, c->half_cnt, c->full_start, c->half_start, c->full_j,
                                    c->full_ref, c->half_i, c->half_j, g, c->flags);
    cudaMemsetAsync(c->full_cnt, 0, sizeof(int) * n, st);  // reused as the per-row slot counter
    k_transpose_scatter<<<amp_blocks(c->cap_half, 256), 256, 0, st>>>(c->cap_half, c->half_j, c->full_start,
                                                                      c->half_cnt, c->full_cnt, c->tr_tmp, g,
                                                                      c->half_start, c->flags);
    k_transpose_sort<<<lb, 256, 0, st>>>(n, c->full_start, c->half_cnt, c->tr_tmp, c->half_i, c->full_j, c->full_ref,
                                        c->pos_tr, g, c->half_start, c->flags);
  }
  c->n_launch += 1;
  k_list_readback<<<1, 32, 0, st>>>(c->full_start + n, c->half_start + n, c->flags, c->hibuf_d);
  if ((r = cuda_check(c, cudaStreamSynchronize(st), "list count"))) return r;
  if (c->hibuf[2] & 2) return fail(c, AMP_ERR_ARG, "alpha must be > 0 for every site");
  c->n_full = c->hibuf[0];
  c->n_half = c->hibuf[1];
  if (c->n_full != 2 * c->n_half) return fail(c, AMP_ERR_GEOMETRY, "inconsistent neighbour counts");
  if (c->n_full > (1LL << 30)) return fail(c, AMP_ERR_GEOMETRY, "too many pairs");
  if (speculative && !(c->hibuf[2] & (4 | 8))) return AMP_OK;  // filled in place
  if (c->n_full > c->cap_full || c->n_half > c->cap_half) {
    void** bufs[] = {(void**)&c->full_j, (void**)&c->full_ref, (void**)&c->tr_tmp, (void**)&c->half_i, (void**)&c->half_j,
                     (void**)&c->C64, (void**)&c->Ep64, (void**)&c->T32, (void**)&c->Ep32,
                     (void**)&c->pos_tr, (void**)&c->intra};
    for (void** b : bufs) {
      dev_free(c, *b);
      *b = nullptr;
    }
    const long long caph = c->n_half + c->n_half / 4 + 1024, capf = 2 * caph;
    c->cap_half = c->cap_full = 0;
    if ((r = dev_alloc(c, &c->full_j, capf)) || (r = dev_alloc(c, &c->full_ref, capf)) ||
        (r = dev_alloc(c, &c->tr_tmp, capf)) ||
        (r = dev_alloc(c, &c->half_i, caph)) || (r = dev_alloc(c, &c->half_j, caph)) ||
        (r = dev_alloc(c, &c->pos_tr, caph)) || (r = dev_alloc(c, &c->Ep64, 6 * caph)))
      return r;
    if (c->cfg.precision == AMP_FP64) {
      if ((r = dev_alloc(c, &c->C64, capf))) return r;
    } else {
      if ((r = dev_alloc(c, &c->T32, 6 * capf)) || (r = dev_alloc(c, &c->Ep32, 6 * caph))) return r;
    }
    if ((r = dev_alloc(c, &c->intra, caph + 1))) return r;
    c->cap_half = caph;
    c->cap_full = capf;
  }
  if (c->hibuf[2] & 4) {  // a slab row overflowed: second pass over the same candidates
    if (from_candidates)
      k_filter<1><<<lb, 256, 0, st>>>(P, c->pos32, c->atomA, c->cand_start, c->cand_j, nullptr, nullptr,
                                      c->full_start, c->half_start, c->full_j, c->full_ref, c->half_i, c->half_j,
                                      nullptr, nullptr);
    else
      k_neighbours<1><<<lb, 256, 0, st>>>(P, c->pos32, c->atomA, c->slot_tmp, c->cell_start, nullptr, nullptr,
                                          c->full_start, c->half_start, c->full_j, c->full_ref, c->half_i,
                                          c->half_j, nullptr, nullptr);
  } else {
    k_slab_copy<<<lb, 256, 0, st>>>(n, slab, c->slab, c->half_cnt, c->full_start, c->half_start, c->full_j,
                                    c->full_ref, c->half_i, c->half_j, none, c->flags);
  }
  cudaMemsetAsync(c->full_cnt, 0, sizeof(int) * n, st);  // reused as the per-row slot counter
  k_transpose_scatter<<<amp_blocks(c->n_half, 256), 256, 0, st>>>(c->n_half, c->half_j, c->full_start, c->half_cnt,
                                                                  c->full_cnt, c->tr_tmp, none, c->half_start,
                                                                  c->flags);
  k_transpose_sort<<<lb, 256, 0, st>>>(n, c->full_start, c->half_cnt, c->tr_tmp, c->half_i, c->full_j, c->full_ref,
                                      c->pos_tr, none, c->half_start, c->flags);
  return cuda_check(c, cudaGetLastError(), "list fill launch");
}

}  // namespace

// Exact lists (cutoff) from the stored candidates (cutoff + skin).
int filter_lists(amp_ctx* c) {
  ListParams P;
  int r;
  if ((r = list_params(c, c->cfg.cutoff, &P))) return r;
  c->n_launch += 6;
  cudaMemsetAsync(c->flags, 0, sizeof(int), c->stream);  // flags[3] (a displacement) is kept
  k_filter<2><<<amp_blocks((long long)c->n * 32, 256), 256, 0, c->stream>>>(
      P, c->pos32, c->atomA, c->cand_start, c->cand_j, c->full_cnt, c->half_cnt, nullptr, nullptr, nullptr, nullptr,
      nullptr, nullptr, c->slab, c->flags);
  return finish_lists(c, P, true);
}

int build_cells_and_lists(amp_ctx* c, const double* xyz, const double* q, const double* dip,
                          const double* quad, const double* alpha, const double* thole, const int* mol) {
  const int n = c->n;
  const double L = c->cfg.box, rc = c->cfg.cutoff;
  // with a skin the cell search collects the candidates within rc + skin
  const double skin = c->skin, rlist = rc + skin;
  cudaStream_t st = c->stream;
  // cells of edge >= rlist / 2 (the neighbour search spans two cells per axis)
  int nc = (int)floor(2.0 * L / (rlist + 1e-6));
  if (nc < 1) nc = 1;
  if (nc > 1024) nc = 1024;
  const int ncell = nc * nc * nc;
  if (ncell > c->ncell_cap) {
    dev_free(c, c->cell_count);
    dev_free(c, c->cell_start);
    dev_free(c, c->cell_fill);
    c->cell_count = c->cell_start = c->cell_fill = nullptr;
    int r;
    if ((r = dev_alloc(c, &c->cell_count, ncell)) || (r = dev_alloc(c, &c->cell_start, ncell + 1)) ||
        (r = dev_alloc(c, &c->cell_fill, ncell)))
      return r;
    c->ncell_cap = ncell;
  }
  c->nc = nc;
  c->ncell = ncell;
  c->skin_built = 0.0;
  int r;
  if ((r = cuda_check(c, cudaMemsetAsync(c->cell_count, 0, sizeof(int) * ncell, st), "memset")) ||
      (r = cuda_check(c, cudaMemsetAsync(c->cell_fill, 0, sizeof(int) * ncell, st), "memset")) ||
      (r = cuda_check(c, cudaMemsetAsync(c->flags, 0, sizeof(int) * 4, st), "memset")))
    return r;
  c->n_launch += 6;  // cell_assign .. k_neighbours below
  k_cell_assign<<<amp_blocks(n, 256), 256, 0, st>>>(n, xyz, L, nc, c->cell_of, c->cell_count);
  k_scan_exclusive<<<1, 1024, 0, st>>>(c->cell_count, c->cell_start, ncell);
  k_cell_scatter<<<amp_blocks(n, 256), 256, 0, st>>>(n, c->cell_of, c->cell_start, c->cell_fill, c->slot_tmp);
  k_cell_sort<<<amp_blocks((long long)ncell * 32, 256), 256, 0, st>>>(ncell, c->cell_start, c->slot_tmp, c->perm);
  k_gather_atoms<<<amp_blocks(n, 256), 256, 0, st>>>(n, c->perm, xyz, q, dip, quad, alpha, thole, mol, L,
                                                     c->inv_perm, c->atomA, c->atomB, c->atomC, c->atomD,
                                                     c->pos32, c->cell_of, c->slot_tmp, c->alph, c->flags);
  // the atom records in cell order are complete: the reciprocal-space work of
  // the geometry starts on the side stream, beside the neighbour search
  if ((r = pme_geometry(c))) return r;
  ListParams P;
  if ((r = list_params(c, rlist, &P))) return r;
  const int lb = amp_blocks((long long)n * 32, 256);
  {
    PhaseScope ps(c, AMP_PHASE_LIST_SEARCH);
    k_neighbours<2><<<lb, 256, 0, st>>>(P, c->pos32, c->atomA, c->slot_tmp, c->cell_start, c->full_cnt,
                                        c->half_cnt, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, c->slab,
                                        c->flags);
  }
  c->n_launch += 4;  // scan .. transpose_sort
  if ((r = finish_lists(c, P, false))) return r;
  if (skin <= 0.0) return AMP_OK;
  // keep the candidates (rows of the list within rc + skin) and the positions
  // they were found at, then filter the exact lists out of them
  if (n + 1 > c->cand_start_cap) {
    dev_free(c, c->cand_start);
    dev_free(c, c->xref);
    dev_free(c, c->abak);
    dev_free(c, c->pbak);
    c->cand_start = nullptr;
    c->xref = c->abak = nullptr;
    c->pbak = nullptr;
    c->cand_start_cap = 0;
    if ((r = dev_alloc(c, &c->cand_start, (long long)n + 1)) || (r = dev_alloc(c, &c->xref, (long long)n)) ||
        (r = dev_alloc(c, &c->abak, (long long)n)) || (r = dev_alloc(c, &c->pbak, (long long)n)))
      return r;
    c->cand_start_cap = n + 1;
  }
  if (c->n_full > c->cand_cap) {
    dev_free(c, c->cand_j);
    c->cand_j = nullptr;
    c->cand_cap = 0;
    const long long cap = c->n_full + c->n_full / 4 + 1024;
    if ((r = dev_alloc(c, &c->cand_j, cap))) return r;
    c->cand_cap = cap;
  }
  cudaMemcpyAsync(c->cand_start, c->full_start, sizeof(int) * (n + 1), cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(c->cand_j, c->full_j, sizeof(int) * c->n_full, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(c->xref, c->atomA, sizeof(double4_32a) * n, cudaMemcpyDeviceToDevice, st);
  if ((r = filter_lists(c))) return r;
  c->skin_built = skin;
  return AMP_OK;
}

// New positions for the current atoms: true in *reused if no atom moved more
// than skin/2 (minimum image) since the candidates were found; then the exact
// lists are filtered out of them (the pair terms and PME weights are the
// caller's next steps). The positions are applied and filtered at once, the
// largest displacement read with the list counts (one host round trip); if it
// is too large, the previous positions and their lists are put back and
// *reused is false (a second round trip, the rare case).
int reuse_lists(amp_ctx* c, const double* xyz, bool* reused) {
  *reused = false;
  if (c->skin_built <= 0.0) return AMP_OK;
  const int n = c->n;
  cudaStream_t st = c->stream;
  int r;
  if ((r = cuda_check(c, cudaMemsetAsync(c->flags + 3, 0, sizeof(int), st), "memset"))) return r;
  c->n_launch += 2;
  k_displacement<<<amp_blocks(n, 256), 256, 0, st>>>(n, c->perm, xyz, c->xref, c->cfg.box, c->flags + 3);
  cudaMemcpyAsync(c->abak, c->atomA, sizeof(double4_32a) * n, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(c->pbak, c->pos32, sizeof(float4) * n, cudaMemcpyDeviceToDevice, st);
  k_apply_positions<<<amp_blocks(n, 256), 256, 0, st>>>(n, c->perm, xyz, c->cfg.box, c->atomA, c->pos32);
  if ((r = filter_lists(c))) return r;
  float d2;
  std::memcpy(&d2, &c->hibuf[5], sizeof d2);  // flags[3], read with the counts
  const double half = 0.5 * c->skin_built;
  // the float maximum is rounded: keep a relative margin below (skin/2)^2
  if ((double)d2 <= half * half * (1.0 - 1e-5)) {
    *reused = true;
    return AMP_OK;
  }
  cudaMemcpyAsync(c->atomA, c->abak, sizeof(double4_32a) * n, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(c->pos32, c->pbak, sizeof(float4) * n, cudaMemcpyDeviceToDevice, st);
  return filter_lists(c);
}

}  // namespace amp
