// Divide-and-conquer Jacobi iterations (DC-JI) on the GPU.
//
// The paper's outlook (Section "Perspectives on Tinker-HP 1.2 performance")
// names DC-JI (Nocito & Beran, 2018) as the polarization solver of the outer
// level of its multi-timestep integrator. Reading used here (the same as the
// oracle's): the sites are split into blocks of whole molecules; every
// iteration solves each block's own equations exactly, with the other
// blocks' dipoles from the previous iteration,
//   A_BB mu_B^(k+1) = E_B - sum_{C != B} A_BC mu_C^(k),   mu^(0) = alpha E,
// i.e. mu <- mu + D^-1 (E - A mu) with D the block diagonal of
// A = diag(1/alpha) - T, and stops when 4.8032047 sqrt(sum |alpha r_i|^2 / N)
// < tol (r = E - A mu), the solver's criterion.
//
// D is the exact block diagonal of the context's operator (real space,
// reciprocal space and self term): column (a, c) of A is A e_(a,c), one
// operator application per column, restricted to the rows of a's block. So
// the assembly costs 3N applications and the method, as in the oracle, is
// for small systems. The blocks are symmetrised ((D + D^T)/2, which the
// operator is up to rounding), factorised by Cholesky in float64 (one CTA per
// block) and every iteration takes one operator application for the residual
// and one forward and one backward substitution per block (one CTA each).
#include <vector>

#include "amp_internal.cuh"

namespace amp {
namespace {

constexpr int kBlockThreads = 256;

// e = unit vector of sorted atom a, component k
__global__ void k_unit(int n, int a, int k, double4_32a* __restrict__ v) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  v[s] = make_double4_32a(s == a && k == 0 ? 1.0 : 0.0, s == a && k == 1 ? 1.0 : 0.0, s == a && k == 2 ? 1.0 : 0.0,
                          0.0);
}

// Column (la, k) of block b's matrix: rows (ls, r) for the block's atoms s,
// A[(ls, r), (la, k)] = [s == a, r == k] / alpha_s - (T e)_(s, r).
__global__ void k_column(int b, int a, int k, const int* __restrict__ bstart, const int* __restrict__ batoms,
                         const int* __restrict__ loc, const long long* __restrict__ moff,
                         const double2* __restrict__ al, const double4_32a* __restrict__ t, double* __restrict__ M) {
  const int s0 = bstart[b], nb = bstart[b + 1] - s0, m = 3 * nb;
  const int col = 3 * loc[a] + k;
  double* A = M + moff[b];
  for (int q = threadIdx.x; q < m; q += blockDim.x) {
    const int ls = q / 3, r = q - 3 * ls, s = batoms[s0 + ls];
    const double* ts = reinterpret_cast<const double*>(t + s);
    A[(long long)q * m + col] = (s == a && r == k ? al[s].y : 0.0) - ts[r];
  }
}

// Symmetrise and factorise each block in place (lower triangle L, row-major,
// A = L L^T), float64, one CTA per block. bad[0] = 1 + block if a pivot is
// not positive.
__global__ void __launch_bounds__(kBlockThreads) k_cholesky(const int* __restrict__ bstart,
                                                            const long long* __restrict__ moff,
                                                            double* __restrict__ M, int* __restrict__ bad) {
  const int b = blockIdx.x, m = 3 * (bstart[b + 1] - bstart[b]);
  double* A = M + moff[b];
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int i = e / m, j = e - i * m;
    if (i > j) {
      const double v = 0.5 * (A[(long long)i * m + j] + A[(long long)j * m + i]);
      A[(long long)i * m + j] = v;
      A[(long long)j * m + i] = v;
    }
  }
  __syncthreads();
  __shared__ double piv;
  for (int k = 0; k < m; ++k) {
    if (threadIdx.x == 0) {
      const double d = A[(long long)k * m + k];
      if (!(d > 0.0)) {
        atomicCAS(bad, 0, 1 + b);
        piv = 1.0;
      } else {
        piv = sqrt(d);
      }
      A[(long long)k * m + k] = piv;
    }
    __syncthreads();
    const double inv = 1.0 / piv;
    for (int i = k + 1 + threadIdx.x; i < m; i += blockDim.x) A[(long long)i * m + k] *= inv;
    __syncthreads();
    // trailing update of the lower triangle: A[i][j] -= L[i][k] L[j][k], k < j <= i
    const int t = m - k - 1;
    for (int e = threadIdx.x; e < t * t; e += blockDim.x) {
      const int i = k + 1 + e / t, j = k + 1 + e % t;
      if (j <= i) A[(long long)i * m + j] -= A[(long long)i * m + k] * A[(long long)j * m + k];
    }
    __syncthreads();
  }
}

// res = E - A mu = E - mu/alpha + T mu; per-block partial sums of |alpha res|^2
__global__ void __launch_bounds__(kBlockThreads) k_residual(int n, const double4_32a* __restrict__ E,
                                                            const double4_32a* __restrict__ mu,
                                                            const double4_32a* __restrict__ t,
                                                            const double2* __restrict__ al,
                                                            double4_32a* __restrict__ res, double* __restrict__ part) {
  __shared__ double sh[kBlockThreads / 32];
  double zz = 0.0;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n) {
    const double a = al[s].x, ia = al[s].y;
    const double4_32a e = E[s], m = mu[s], tt = t[s];
    const double4_32a r = make_double4_32a(e.x - m.x * ia + tt.x, e.y - m.y * ia + tt.y, e.z - m.z * ia + tt.z, 0.0);
    res[s] = r;
    zz = a * a * (r.x * r.x + r.y * r.y + r.z * r.z);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) zz += __shfl_xor_sync(0xffffffffu, zz, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = zz;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int w = 0; w < kBlockThreads / 32; ++w) tot += sh[w];
    part[blockIdx.x] = tot;
  }
}

// RMS (Debye) of alpha res from the partials, fixed order, into out[0]
__global__ void k_rms(int nparts, int n, const double* __restrict__ part, double* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double tot = 0.0;
  for (int k = 0; k < nparts; ++k) tot += part[k];
  out[0] = kDebye * sqrt(tot / (double)(n > 0 ? n : 1));
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < kBlockThreads / 32; ++w) s += sh[w];
  return s;  // every thread, the same fixed order
}

// One CTA per block: delta = L^-T L^-1 res_B (forward, then backward
// substitution; y kept in delta's storage), mu_B += delta.
__global__ void __launch_bounds__(kBlockThreads) k_block_update(const int* __restrict__ bstart,
                                                                const int* __restrict__ batoms,
                                                                const long long* __restrict__ moff,
                                                                const double* __restrict__ M,
                                                                const double4_32a* __restrict__ res,
                                                                double* __restrict__ work,
                                                                double4_32a* __restrict__ mu) {
  __shared__ double sh[kBlockThreads / 32];
  const int b = blockIdx.x, s0 = bstart[b], m = 3 * (bstart[b + 1] - s0);
  const double* L = M + moff[b];
  double* y = work + 3LL * s0;
  for (int q = threadIdx.x; q < m; q += blockDim.x)
    y[q] = reinterpret_cast<const double*>(res + batoms[s0 + q / 3])[q % 3];
  __syncthreads();
  for (int i = 0; i < m; ++i) {  // L y = r
    double p = 0.0;
    for (int k = threadIdx.x; k < i; k += blockDim.x) p += L[(long long)i * m + k] * y[k];
    p = block_sum(p, sh);
    if (threadIdx.x == 0) y[i] = (y[i] - p) / L[(long long)i * m + i];
    __syncthreads();
  }
  for (int i = m - 1; i >= 0; --i) {  // L^T d = y
    double p = 0.0;
    for (int k = i + 1 + threadIdx.x; k < m; k += blockDim.x) p += L[(long long)k * m + i] * y[k];
    p = block_sum(p, sh);
    if (threadIdx.x == 0) y[i] = (y[i] - p) / L[(long long)i * m + i];
    __syncthreads();
  }
  for (int q = threadIdx.x; q < m; q += blockDim.x) reinterpret_cast<double*>(mu + batoms[s0 + q / 3])[q % 3] += y[q];
}

__global__ void k_alpha_e(int n, const double4_32a* __restrict__ E, const double2* __restrict__ al,
                          double4_32a* __restrict__ mu) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const double a = al[s].x;
  const double4_32a e = E[s];
  mu[s] = make_double4_32a(a * e.x, a * e.y, a * e.z, 0.0);
}

}  // namespace

// t = T v (the context's float64-path operator; v split into the operator's
// input buffers first)
static int apply_T_f64(amp_ctx* c, const double4_32a* v, double4_32a* t) {
  launch_split(c, v, c->p32, c->plo);
  return apply_T_sorted(c, v, c->p32, c->plo, t, nullptr);
}

static int dcji(amp_ctx* c, const double* E0, const int* block_of, int n_blocks, double tol, int max_iter,
                double* mu_out, int* iters, double* rms_out) {
  const int n = c->n;
  cudaStream_t st = c->stream;
  int r;
  // blocks in sorted order: each block's atoms by caller index
  std::vector<int> perm(n);
  if ((r = cuda_check(c, cudaMemcpyAsync(perm.data(), c->perm, sizeof(int) * n, cudaMemcpyDeviceToHost, st),
                      "perm read")) ||
      (r = cuda_check(c, cudaStreamSynchronize(st), "perm read")))
    return r;
  std::vector<int> inv(n);
  for (int s = 0; s < n; ++s) inv[perm[s]] = s;
  std::vector<int> cnt(n_blocks, 0);
  for (int i = 0; i < n; ++i) ++cnt[block_of[i]];
  std::vector<int> bstart(n_blocks + 1, 0);
  for (int b = 0; b < n_blocks; ++b) {
    if (cnt[b] == 0) return fail(c, AMP_ERR_ARG, "amp_dcji: block %d is empty", b);
    bstart[b + 1] = bstart[b] + cnt[b];
  }
  std::vector<int> fill(bstart.begin(), bstart.end() - 1), batoms(n), loc(n), blk(n);
  for (int i = 0; i < n; ++i) {  // caller order within a block
    const int b = block_of[i], s = inv[i];
    loc[s] = fill[b] - bstart[b];
    blk[s] = b;
    batoms[fill[b]++] = s;
  }
  std::vector<long long> moff(n_blocks + 1, 0);
  for (int b = 0; b < n_blocks; ++b) moff[b + 1] = moff[b] + 9LL * cnt[b] * cnt[b];
  // device buffers (freed at the end of the call)
  int *d_bstart = nullptr, *d_batoms = nullptr, *d_loc = nullptr, *d_bad = nullptr;
  long long* d_moff = nullptr;
  double *d_M = nullptr, *d_work = nullptr, *d_part = nullptr, *d_rms = nullptr;
  double4_32a *E = nullptr, *mu = nullptr, *t = nullptr, *res = nullptr, *e = nullptr;
  const int nb = amp_blocks(n, kBlockThreads);
  auto cleanup = [&]() {
    for (void* p : {(void*)d_bstart, (void*)d_batoms, (void*)d_loc, (void*)d_bad, (void*)d_moff, (void*)d_M,
                    (void*)d_work, (void*)d_part, (void*)d_rms, (void*)E, (void*)mu, (void*)t, (void*)res, (void*)e})
      dev_free(c, p);
  };
  if ((r = dev_alloc(c, &d_bstart, n_blocks + 1)) || (r = dev_alloc(c, &d_batoms, n)) ||
      (r = dev_alloc(c, &d_loc, n)) || (r = dev_alloc(c, &d_bad, 1)) || (r = dev_alloc(c, &d_moff, n_blocks + 1)) ||
      (r = dev_alloc(c, &d_M, moff[n_blocks])) || (r = dev_alloc(c, &d_work, 3LL * n)) ||
      (r = dev_alloc(c, &d_part, nb)) || (r = dev_alloc(c, &d_rms, 1)) || (r = dev_alloc(c, &E, n)) ||
      (r = dev_alloc(c, &mu, n)) || (r = dev_alloc(c, &t, n)) || (r = dev_alloc(c, &res, n)) ||
      (r = dev_alloc(c, &e, n))) {
    cleanup();
    return r;
  }
  cudaMemcpyAsync(d_bstart, bstart.data(), sizeof(int) * (n_blocks + 1), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(d_batoms, batoms.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(d_loc, loc.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(d_moff, moff.data(), sizeof(long long) * (n_blocks + 1), cudaMemcpyHostToDevice, st);
  cudaMemsetAsync(d_bad, 0, sizeof(int), st);
  launch_to_sorted(c, E0, E);
  c->n_launch += 1;
  // the block diagonal of A, one operator application per column
  for (int a = 0; a < n && !r; ++a)
    for (int k = 0; k < 3 && !r; ++k) {
      c->n_launch += 2;
      k_unit<<<nb, kBlockThreads, 0, st>>>(n, a, k, e);
      if ((r = apply_T_f64(c, e, t))) break;
      k_column<<<1, kBlockThreads, 0, st>>>(blk[a], a, k, d_bstart, d_batoms, d_loc, d_moff, c->alph, t, d_M);
    }
  if (!r) {
    c->n_launch += 2;
    k_cholesky<<<n_blocks, kBlockThreads, 0, st>>>(d_bstart, d_moff, d_M, d_bad);
    k_alpha_e<<<nb, kBlockThreads, 0, st>>>(n, E, c->alph, mu);
    int bad = 0;
    if (!(r = cuda_check(c, cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, st), "dcji")) &&
        !(r = cuda_check(c, cudaStreamSynchronize(st), "dcji factorisation")) && bad)
      r = fail(c, AMP_ERR_NOT_CONVERGED, "amp_dcji: block %d is not positive definite", bad - 1);
  }
  int it = 0;
  double rms = 0.0;
  while (!r) {
    if ((r = apply_T_f64(c, mu, t))) break;
    c->n_launch += 2;
    k_residual<<<nb, kBlockThreads, 0, st>>>(n, E, mu, t, c->alph, res, d_part);
    k_rms<<<1, 32, 0, st>>>(nb, n, d_part, d_rms);
    if ((r = cuda_check(c, cudaMemcpyAsync(&rms, d_rms, sizeof(double), cudaMemcpyDeviceToHost, st), "dcji")) ||
        (r = cuda_check(c, cudaStreamSynchronize(st), "dcji residual")))
      break;
    if (!(rms >= tol) || it >= max_iter) break;
    c->n_launch += 1;
    k_block_update<<<n_blocks, kBlockThreads, 0, st>>>(d_bstart, d_batoms, d_moff, d_M, res, d_work, mu);
    ++it;
  }
  if (!r) {
    launch_from_sorted(c, mu, mu_out);
    r = cuda_check(c, cudaStreamSynchronize(st), "dcji");
  }
  cleanup();
  if (r) return r;
  if (iters) *iters = it;
  if (rms_out) *rms_out = rms;
  return AMP_OK;
}

}  // namespace amp

extern "C" int amp_dcji(amp_ctx* c, const double* E0, const int* block_of, int n_blocks, double tol_debye,
                        int max_iter, double* mu, int* iters, double* rms_debye) {
  using namespace amp;
  if (!c) return AMP_ERR_ARG;
  join_geometry(c);
  if (!c->have_system) return fail(c, AMP_ERR_STATE, "no system set");
  if (!E0 || !mu || !block_of) return fail(c, AMP_ERR_ARG, "amp_dcji: E0, mu and block_of are required");
  if (c->cfg.precision != AMP_FP64) return fail(c, AMP_ERR_ARG, "amp_dcji: float64 contexts only");
  if (n_blocks < 1 || n_blocks > c->n) return fail(c, AMP_ERR_ARG, "amp_dcji: n_blocks must be in [1, N]");
  if (!(tol_debye >= 0.0) || max_iter < 0) return fail(c, AMP_ERR_ARG, "amp_dcji: bad tolerance or max_iter");
  for (int i = 0; i < c->n; ++i)
    if (block_of[i] < 0 || block_of[i] >= n_blocks)
      return fail(c, AMP_ERR_ARG, "amp_dcji: block_of[%d] = %d is outside [0, %d)", i, block_of[i], n_blocks);
  return dcji(c, E0, block_of, n_blocks, tol_debye, max_iter, mu, iters, rms_debye);
}
