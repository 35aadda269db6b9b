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
//   4. count pass: one warp per atom, candidates from the (distinct) 27
//      neighbour cells, float32 distance pre-filter with a margin, exact
//      float64 decision d.d < rc^2 for candidates near the cutoff;
//   5. scan the row counts; fill pass writes the full rows and the half rows;
//   6. each pair id is scattered to its non-owner's row, which sorts that part
//      of the row by pair id (deterministic order).
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

// Single-block exclusive scan: out[k] = sum_{m<k} in[k], out[n] = total.
__global__ void k_scan_exclusive(const int* __restrict__ in, int* __restrict__ out, int n) {
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
  int n, nc, nof;
  double L, rc2;
  float Lf, invLf, lo2, hi2;
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

template <bool kFill>
__global__ void k_neighbours(ListParams P, const float4* __restrict__ pos32, const double4_32a* __restrict__ A,
                             const int* __restrict__ cell_sorted, const int* __restrict__ cell_start, int* __restrict__ full_cnt,
                             int* __restrict__ half_cnt, const int* __restrict__ full_start,
                             const int* __restrict__ half_start, int* __restrict__ full_j,
                             int* __restrict__ full_ref, int* __restrict__ half_i, int* __restrict__ half_j) {
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= P.n) return;
  const unsigned lt = (1u << lane) - 1u;
  const float4 pi = pos32[i];
  const double4_32a ai = A[i];
  const int cself = cell_sorted[i];  // the cell the atom was binned in (float64 wrap)
  const int ci[3] = {cself / (P.nc * P.nc), (cself / P.nc) % P.nc, cself % P.nc};
  int nfull = 0, nhalf = 0;
  const int fbase = kFill ? full_start[i] : 0;
  const int hbase = kFill ? half_start[i] : 0;
  for (int ox = 0; ox < P.nof; ++ox) {
    int cx = (ci[0] + (P.nof == 3 ? ox - 1 : ox) + P.nc) % P.nc;
    for (int oy = 0; oy < P.nof; ++oy) {
      int cy = (ci[1] + (P.nof == 3 ? oy - 1 : oy) + P.nc) % P.nc;
      for (int oz = 0; oz < P.nof; ++oz) {
        int cz = (ci[2] + (P.nof == 3 ? oz - 1 : oz) + P.nc) % P.nc;
        int cell = (cx * P.nc + cy) * P.nc + cz;
        int s = cell_start[cell], e = cell_start[cell + 1];
        for (int k0 = s; k0 < e; k0 += 32) {
          int k = k0 + lane;
          bool in = false;
          if (k < e && k != i) {
            float4 pj = pos32[k];
            float dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
            dx -= P.Lf * rintf(dx * P.invLf);
            dy -= P.Lf * rintf(dy * P.invLf);
            dz -= P.Lf * rintf(dz * P.invLf);
            float r2 = dx * dx + dy * dy + dz * dz;
            if (r2 < P.hi2) in = (r2 <= P.lo2) ? true : exact_in_range(ai, A[k], P.L, P.rc2);
          }
          bool own = in && ((i < k) != (((i + k) & 1) != 0));
          unsigned mf = __ballot_sync(0xffffffffu, in);
          unsigned mh = __ballot_sync(0xffffffffu, own);
          if (kFill && own) {
            // owned pairs open the row: full slot and pair id share the rank
            const int rank = nhalf + __popc(mh & lt);
            const int pid = hbase + rank;
            full_j[fbase + rank] = k;
            full_ref[fbase + rank] = pid << 1;
            half_i[pid] = i;
            half_j[pid] = k;
          }
          nfull += __popc(mf);
          nhalf += __popc(mh);
        }
      }
    }
  }
  if (!kFill && lane == 0) {
    full_cnt[i] = nfull;
    half_cnt[i] = nhalf;
  }
}

// The rest of row j lists the pairs owned by other rows: every pair id is
// scattered to its non-owner's row (atomic slot), then each row sorts that part
// by pair id, so the final order does not depend on the atomics.
__global__ void k_transpose_scatter(long long nh, const int* __restrict__ half_j,
                                    const int* __restrict__ full_start, const int* __restrict__ half_cnt,
                                    int* __restrict__ tcount, int* __restrict__ tmp) {
  const long long pid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (pid >= nh) return;
  const int j = half_j[pid];
  const int slot = full_start[j] + half_cnt[j] + atomicAdd(&tcount[j], 1);
  tmp[slot] = (int)pid;
}

__global__ void k_transpose_sort(int n, const int* __restrict__ full_start, const int* __restrict__ half_cnt,
                                 const int* __restrict__ tmp, const int* __restrict__ half_i,
                                 int* __restrict__ full_j, int* __restrict__ full_ref) {
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= n) return;
  const int lo = full_start[i] + half_cnt[i], hi = full_start[i + 1];
  for (int e = lo + lane; e < hi; e += 32) {
    const int p = tmp[e];
    int rank = 0;
    for (int m = lo; m < hi; ++m) rank += tmp[m] < p;
    full_ref[lo + rank] = (p << 1) | 1;
    full_j[lo + rank] = half_i[p];
  }
}

}  // namespace

int build_cells_and_lists(amp_ctx* c, const double* xyz, const double* q, const double* dip,
                          const double* quad, const double* alpha, const double* thole, const int* mol) {
  const int n = c->n;
  const double L = c->cfg.box, rc = c->cfg.cutoff;
  cudaStream_t st = c->stream;
  int nc = (int)floor(L / (rc + 1e-6));
  if (nc < 1) nc = 1;
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
  int r;
  if ((r = cuda_check(c, cudaMemsetAsync(c->cell_count, 0, sizeof(int) * ncell, st), "memset")) ||
      (r = cuda_check(c, cudaMemsetAsync(c->cell_fill, 0, sizeof(int) * ncell, st), "memset")) ||
      (r = cuda_check(c, cudaMemsetAsync(c->flags, 0, sizeof(int) * 4, st), "memset")))
    return r;
  c->n_launch += 11;  // cell_assign .. transpose_sort below
  k_cell_assign<<<amp_blocks(n, 256), 256, 0, st>>>(n, xyz, L, nc, c->cell_of, c->cell_count);
  k_scan_exclusive<<<1, 1024, 0, st>>>(c->cell_count, c->cell_start, ncell);
  k_cell_scatter<<<amp_blocks(n, 256), 256, 0, st>>>(n, c->cell_of, c->cell_start, c->cell_fill, c->slot_tmp);
  k_cell_sort<<<amp_blocks((long long)ncell * 32, 256), 256, 0, st>>>(ncell, c->cell_start, c->slot_tmp, c->perm);
  k_gather_atoms<<<amp_blocks(n, 256), 256, 0, st>>>(n, c->perm, xyz, q, dip, quad, alpha, thole, mol, L,
                                                     c->inv_perm, c->atomA, c->atomB, c->atomC, c->atomD,
                                                     c->pos32, c->cell_of, c->slot_tmp, c->alph, c->flags);
  ListParams P;
  P.n = n;
  P.nc = nc;
  P.nof = nc >= 3 ? 3 : nc;
  P.L = L;
  P.rc2 = rc * rc;
  P.Lf = (float)L;
  P.invLf = (float)(1.0 / L);
  P.lo2 = (float)(rc * rc - 0.01);
  P.hi2 = (float)(rc * rc + 0.01);
  const int lb = amp_blocks((long long)n * 32, 256);
  k_neighbours<false><<<lb, 256, 0, st>>>(P, c->pos32, c->atomA, c->slot_tmp, c->cell_start, c->full_cnt, c->half_cnt,
                                          nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
  k_scan_exclusive<<<1, 1024, 0, st>>>(c->full_cnt, c->full_start, n);
  k_scan_exclusive<<<1, 1024, 0, st>>>(c->half_cnt, c->half_start, n);
  if ((r = cuda_check(c, cudaGetLastError(), "list count launch"))) return r;
  cudaMemcpyAsync(&c->hibuf[0], c->full_start + n, sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(&c->hibuf[1], c->half_start + n, sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(&c->hibuf[2], c->flags, sizeof(int), cudaMemcpyDeviceToHost, st);
  if ((r = cuda_check(c, cudaStreamSynchronize(st), "list count"))) return r;
  if (c->hibuf[2] & 2) return fail(c, AMP_ERR_ARG, "alpha must be > 0 for every site");
  c->n_full = c->hibuf[0];
  c->n_half = c->hibuf[1];
  if (c->n_full != 2 * c->n_half) return fail(c, AMP_ERR_GEOMETRY, "inconsistent neighbour counts");
  if (c->n_full > (1LL << 30)) return fail(c, AMP_ERR_GEOMETRY, "too many pairs");
  if (c->n_full > c->cap_full || c->n_half > c->cap_half) {
    void** bufs[] = {(void**)&c->full_j, (void**)&c->full_ref, (void**)&c->tr_tmp, (void**)&c->half_i, (void**)&c->half_j,
                     (void**)&c->T64, (void**)&c->Ep64, (void**)&c->T32, (void**)&c->Ep32};
    for (void** b : bufs) {
      dev_free(c, *b);
      *b = nullptr;
    }
    const long long caph = c->n_half + c->n_half / 4 + 1024, capf = 2 * caph;
    c->cap_half = c->cap_full = 0;
    if ((r = dev_alloc(c, &c->full_j, capf)) || (r = dev_alloc(c, &c->full_ref, capf)) ||
        (r = dev_alloc(c, &c->tr_tmp, capf)) ||
        (r = dev_alloc(c, &c->half_i, caph)) || (r = dev_alloc(c, &c->half_j, caph)) ||
        (r = dev_alloc(c, &c->Ep64, 6 * caph)))
      return r;
    if (c->cfg.precision == AMP_FP64) {
      if ((r = dev_alloc(c, &c->T64, 6 * caph))) return r;
    } else {
      if ((r = dev_alloc(c, &c->T32, 6 * caph)) || (r = dev_alloc(c, &c->Ep32, 6 * caph))) return r;
    }
    c->cap_half = caph;
    c->cap_full = capf;
  }
  k_neighbours<true><<<lb, 256, 0, st>>>(P, c->pos32, c->atomA, c->slot_tmp, c->cell_start, nullptr, nullptr, c->full_start,
                                         c->half_start, c->full_j, c->full_ref, c->half_i, c->half_j);
  cudaMemsetAsync(c->full_cnt, 0, sizeof(int) * n, st);  // reused as the per-row slot counter
  k_transpose_scatter<<<amp_blocks(c->n_half, 256), 256, 0, st>>>(c->n_half, c->half_j, c->full_start, c->half_cnt,
                                                                  c->full_cnt, c->tr_tmp);
  k_transpose_sort<<<lb, 256, 0, st>>>(n, c->full_start, c->half_cnt, c->tr_tmp, c->half_i, c->full_j, c->full_ref);
  cudaMemcpyAsync(&c->hibuf[2], c->flags, sizeof(int), cudaMemcpyDeviceToHost, st);
  if ((r = cuda_check(c, cudaStreamSynchronize(st), "list fill"))) return r;
  if (c->hibuf[2] & 1) return fail(c, AMP_ERR_GEOMETRY, "neighbour list transpose failed");
  return AMP_OK;
}

}  // namespace amp
