// Truncated conjugate gradient of order one (TCG-1) and its exact gradients.
//
// The paper's outlook (Section "Perspectives on Tinker-HP 1.2 performance")
// names the non-iterative TCG solver (Aviat et al., JCTC 2017) for the
// polarization. TCG-1 is one step of the diagonal-preconditioned CG from the
// direct guess, with the energy of that iterate:
//   u = alpha E,  r = T u (the residual E - A u),  z = alpha r,
//   gamma = (r.z) / (z.A z),  mu_1 = u + gamma z,  U_1 = -1/2 C mu_1 . E.
// mu_1 is not the minimiser, so its gradient runs through gamma, r and z
// (no stationarity shortcut). With w = u.T u (= u.r), s = r.z,
// t = z.A z = s - z.T z, v = alpha T z, dT and dE the derivatives of the
// operator and of the permanent field:
//   dU_1 = -1/2 C [ c.dE + P.dT u + kappa z.dT z ],
//   c = 2 u + (w/t)(2(1-gamma) v + 2 gamma alpha T v) + 2 gamma z,
//   P = 2 (w/t)((1-gamma) z + gamma v) + gamma u,  kappa = gamma w / t
// (a.dT b is symmetric in a and b). The multipoles enter through E only, so
// the moment gradients are those of -1/2 C c.E at fixed c.
//
// On the GPU: three operator applications (T u, T z, T v) in the context's
// working precision, two fixed-order single-block reductions for the
// scalars and the energy, one vector kernel; then the force kernels of
// amp_forces.cu in their bilinear mode: the pair kernel with c (weight 1/2)
// and the pairs (P/2, u), (kappa z/2, z); the reciprocal gradients of c.E
// (weight 1/2) and the Hessian contractions -(a.H_b + b.H_a) of both pairs.
#include "amp_internal.cuh"

namespace amp {
namespace {

constexpr int kRedThreads = 1024;

__device__ __forceinline__ double block_reduce(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = threadIdx.x < kRedThreads / 32 ? sh[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  }
  return s;  // valid in thread 0
}

__device__ __forceinline__ double dot4(const double4_32a& a, const double4_32a& b) {
  return a.x * b.x + a.y * b.y + a.z * b.z;
}

// out = alpha * v
__global__ void k_scale_alpha(int n, const double2* __restrict__ al, const double4_32a* __restrict__ v,
                              double4_32a* __restrict__ out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const double a = al[s].x;
  const double4_32a x = v[s];
  out[s] = make_double4_32a(a * x.x, a * x.y, a * x.z, 0.0);
}

// One block, fixed order: w = u.r, s = r.z, zy = z.y; then
// t = s - zy, gamma = s / t, a = w / t, kappa = gamma w / t into sc[0..5]
// (w, s, t, gamma, a, kappa); sc[6] = 1 if t <= 0 (not positive definite).
__global__ void __launch_bounds__(kRedThreads) k_tcg_scalars(int n, const double4_32a* __restrict__ u,
                                                             const double4_32a* __restrict__ r,
                                                             const double4_32a* __restrict__ z,
                                                             const double4_32a* __restrict__ y,
                                                             double* __restrict__ sc) {
  __shared__ double sh[kRedThreads / 32];
  double w = 0.0, s = 0.0, zy = 0.0;
  for (int k = threadIdx.x; k < n; k += kRedThreads) {
    const double4_32a rk = r[k], zk = z[k];
    w += dot4(u[k], rk);
    s += dot4(rk, zk);
    zy += dot4(zk, y[k]);
  }
  w = block_reduce(w, sh);
  s = block_reduce(s, sh);
  zy = block_reduce(zy, sh);
  if (threadIdx.x == 0) {
    const double t = s - zy, gamma = s / t;
    sc[0] = w;
    sc[1] = s;
    sc[2] = t;
    sc[3] = gamma;
    sc[4] = w / t;
    sc[5] = gamma * w / t;
    sc[6] = t > 0.0 ? 0.0 : 1.0;
  }
}

// mu_1 = u + gamma z; c; P/2; kappa z/2 (the scaled vectors of the bilinear
// pairs), from the scalars of k_tcg_scalars.
__global__ void k_tcg_vectors(int n, const double* __restrict__ sc, const double2* __restrict__ al,
                              const double4_32a* __restrict__ u, const double4_32a* __restrict__ z,
                              const double4_32a* __restrict__ v, const double4_32a* __restrict__ Tv,
                              double4_32a* __restrict__ mu1, double4_32a* __restrict__ cv,
                              double4_32a* __restrict__ ph, double4_32a* __restrict__ zh) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const double gamma = sc[3], a = sc[4], kappa = sc[5], alpha = al[s].x;
  const double4_32a uu = u[s], zz = z[s], vv = v[s], tv = Tv[s];
  const double cu = 2.0, cvv = 2.0 * a * (1.0 - gamma), ctv = 2.0 * a * gamma * alpha, cz = 2.0 * gamma;
  mu1[s] = make_double4_32a(uu.x + gamma * zz.x, uu.y + gamma * zz.y, uu.z + gamma * zz.z, 0.0);
  cv[s] = make_double4_32a(cu * uu.x + cvv * vv.x + ctv * tv.x + cz * zz.x,
                           cu * uu.y + cvv * vv.y + ctv * tv.y + cz * zz.y,
                           cu * uu.z + cvv * vv.z + ctv * tv.z + cz * zz.z, 0.0);
  // P/2 = (w/t)((1-gamma) z + gamma v) + gamma u / 2
  const double pz = a * (1.0 - gamma), pv = a * gamma, pu = 0.5 * gamma;
  ph[s] = make_double4_32a(pz * zz.x + pv * vv.x + pu * uu.x, pz * zz.y + pv * vv.y + pu * uu.y,
                           pz * zz.z + pv * vv.z + pu * uu.z, 0.0);
  const double hk = 0.5 * kappa;
  zh[s] = make_double4_32a(hk * zz.x, hk * zz.y, hk * zz.z, 0.0);
}

// U_1 = -1/2 C mu_1 . E (one block, fixed order) into sc[7]
__global__ void __launch_bounds__(kRedThreads) k_tcg_energy(int n, const double4_32a* __restrict__ mu1,
                                                            const double4_32a* __restrict__ E,
                                                            double* __restrict__ sc) {
  __shared__ double sh[kRedThreads / 32];
  double e = 0.0;
  for (int k = threadIdx.x; k < n; k += kRedThreads) e += dot4(mu1[k], E[k]);
  e = block_reduce(e, sh);
  if (threadIdx.x == 0) sc[7] = -0.5 * kCoulomb * e;
}

}  // namespace

// One operator application t = T v in the working precision (the split of v
// through the operator-input buffers).
static int apply_T_work(amp_ctx* c, const double4_32a* v, double4_32a* t) {
  float4* lo = c->cfg.precision == AMP_MIXED ? nullptr : c->plo;
  launch_split(c, v, c->p32, lo);
  return apply_T_sorted(c, v, c->p32, lo, t, nullptr);
}

int tcg1(amp_ctx* c, const double* E0, double* mu, double* U, double* F, double* gq, double* gd, double* gt) {
  const int n = c->n;
  int r;
  if ((long long)c->tcg_cap < 10LL * n) {
    dev_free(c, c->tcg);
    c->tcg = nullptr;
    c->tcg_cap = 0;
    if ((r = dev_alloc(c, &c->tcg, 10LL * n))) return r;
    c->tcg_cap = 10LL * n;
  }
  if (!c->tcg_sc && (r = dev_alloc(c, &c->tcg_sc, 8))) return r;
  double4_32a *u = c->tcg, *rr = u + n, *z = rr + n, *y = z + n, *v = y + n, *Tv = v + n;
  double4_32a *cv = Tv + n, *ph = cv + n, *zh = ph + n;
  double4_32a* E = c->E0s;
  cudaStream_t st = c->stream;
  const int nb = amp_blocks(n, 256);
  launch_to_sorted(c, E0, E);
  c->n_launch += 2;
  k_scale_alpha<<<nb, 256, 0, st>>>(n, c->alph, E, u);                                // u = alpha E
  if ((r = apply_T_work(c, u, rr))) return r;                                          // r = T u
  k_scale_alpha<<<nb, 256, 0, st>>>(n, c->alph, rr, z);                               // z = alpha r
  if ((r = apply_T_work(c, z, y))) return r;                                           // y = T z
  c->n_launch += 1;
  k_scale_alpha<<<nb, 256, 0, st>>>(n, c->alph, y, v);                                // v = alpha T z
  if ((r = apply_T_work(c, v, Tv))) return r;                                          // T v
  c->n_launch += 3;
  k_tcg_scalars<<<1, kRedThreads, 0, st>>>(n, u, rr, z, y, c->tcg_sc);
  k_tcg_vectors<<<nb, 256, 0, st>>>(n, c->tcg_sc, c->alph, u, z, v, Tv, c->mu, cv, ph, zh);
  k_tcg_energy<<<1, kRedThreads, 0, st>>>(n, c->mu, E, c->tcg_sc);
  if (mu) launch_from_sorted(c, c->mu, mu);
  if (F && (r = bilinear_forces(c, cv, 0.5, ph, u, zh, z, F, gq, gd, gt, nullptr, 0.0))) return r;
  if ((r = cuda_check(c, cudaGetLastError(), "tcg1 launch"))) return r;
  cudaMemcpyAsync(c->hbuf, c->tcg_sc, sizeof(double) * 8, cudaMemcpyDeviceToHost, st);
  if ((r = cuda_check(c, cudaStreamSynchronize(st), "tcg1"))) return r;
  if (c->hbuf[6] != 0.0) return fail(c, AMP_ERR_NOT_CONVERGED, "TCG-1: z.A z <= 0 (operator not positive definite)");
  if (U) *U = c->hbuf[7];
  return AMP_OK;
}

}  // namespace amp

extern "C" int amp_tcg1(amp_ctx* c, const double* E0, double* mu, double* U, double* F, double* gq, double* gdip,
                        double* gquad) {
  using namespace amp;
  if (!c) return AMP_ERR_ARG;
  join_geometry(c);
  if (!c->have_system) return fail(c, AMP_ERR_STATE, "no system set");
  if (!E0) return fail(c, AMP_ERR_ARG, "E0 is null");
  if (c->cluster && F) return fail(c, AMP_ERR_ARG, "amp_tcg1: gradients only for periodic contexts");
  if (!F && (gq || gdip || gquad)) return fail(c, AMP_ERR_ARG, "amp_tcg1: moment gradients need F");
  return tcg1(c, E0, mu, U, F, gq, gdip, gquad);
}
