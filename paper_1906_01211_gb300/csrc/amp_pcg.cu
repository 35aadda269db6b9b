// Preconditioned conjugate gradients on (1/alpha - T) mu = E0 (kernel d).
//
// The paper's solver applies T*mu about nine times per step (Section
// "Sequential performance") and names only "the convergence method"
// (Section "Hotspots"). The method here is CG with the diagonal preconditioner
// M = diag(alpha) (Saad, Algorithm 9.1):
//   r = E0 - A mu; z = alpha r; p = z;
//   loop: q = A p; gamma = r.z / p.q; mu += gamma p; r -= gamma q; z = alpha r;
//         stop if DEBYE sqrt(sum |z_i|^2 / N) < tol;
//         beta = (r.z)_new / (r.z)_old; p = z + beta p.
// It is run in the Chronopoulos-Gear arrangement (J. Comput. Appl. Math. 25,
// 1989), which takes the same steps in exact arithmetic but needs one global
// reduction per iteration instead of two: the operator is applied to z,
// w = A z, and q = A p follows by recurrence:
//   rho = r.z, m = z.w; beta = rho / rho_old (0 at the first step);
//   gamma = rho / (m - beta rho / gamma_old)  [= r.z / p.q];
//   p = z + beta p; q = w + beta q; mu += gamma p; r -= gamma q; z = alpha r.
// On a GPU where a grid-wide synchronisation costs as much as a launch
// (~2.5 us), this leaves two small kernels per iteration after the operator:
// k_cg_dots (w, partial r.z and z.w) and k_cg_step (the update, the new z's
// float split for the operator, and the convergence test by the last block
// to finish). All scalars stay on the device in float64 and partial sums are
// reduced in a fixed order (deterministic). Every kernel of an iteration,
// those of the operator included, returns at once when the device "stop"
// flag is set, so the host can enqueue several iterations between flag reads
// without paying for the ones after convergence.
#include <algorithm>

#include "amp_internal.cuh"

namespace amp {
namespace {

constexpr int kPcgChunk = 4;  // iterations enqueued per flag read after the first chunk
constexpr int NT = kReduceThreads;
constexpr int NB = kReduceBlocks;

// Blocks of a vector kernel over n atoms: one element per thread up to NB
// blocks (grid-stride beyond). Blocks without elements would still pay for
// their float64 reductions, each warp instruction of which holds the float64
// pipe for ~64 cycles on this GPU.
__host__ __device__ __forceinline__ int vec_blocks(int n) {
  const int b = (n + NT - 1) / NT;
  return b < 1 ? 1 : (b > NB ? NB : b);
}

// iflags: [0] stop, [1] iterations done, [2] first step pending (beta = 0),
//         [3] status (0 running, 1 converged, 2 max_iter, 3 breakdown),
//         [4] arrival counter of the last-block reductions
// scal:   [0] rho = r.z of the current z, [1] gamma of the last step,
//         [2] last RMS (Debye), [3] energy
// partials: [0, NB) r.z and [NB, 2 NB) z.w per block (k_cg_dots);
//           [2 NB, 3 NB) z.z per block (k_cg_init, k_cg_step)
enum { F_STOP = 0, F_ITERS = 1, F_FIRST = 2, F_STATUS = 3, F_COUNT = 4 };

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum of two values; result valid in every thread.
__device__ __forceinline__ void block_sum2(double& a, double& b) {
  __shared__ double sa[NT / 32], sb[NT / 32];
  __shared__ double ra, rb;
  a = warp_sum(a);
  b = warp_sum(b);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    sa[w] = a;
    sb[w] = b;
  }
  __syncthreads();
  if (w == 0) {
    double x = l < NT / 32 ? sa[l] : 0.0, y = l < NT / 32 ? sb[l] : 0.0;
    x = warp_sum(x);
    y = warp_sum(y);
    if (l == 0) {
      ra = x;
      rb = y;
    }
  }
  __syncthreads();
  a = ra;
  b = rb;
  __syncthreads();
}

// Every block re-reduces the nb partials in the same order (one warp, then
// broadcast).
__device__ __forceinline__ void reduce_partials(const double* __restrict__ part, int nb, double& a, double& b) {
  __shared__ double ra, rb;
  if (threadIdx.x < 32) {
    double x = 0.0, y = 0.0;
    for (int k = threadIdx.x; k < nb; k += 32) {
      x += part[k];
      y += part[NB + k];
    }
    x = warp_sum(x);
    y = warp_sum(y);
    if (threadIdx.x == 0) {
      ra = x;
      rb = y;
    }
  }
  __syncthreads();
  a = ra;
  b = rb;
  __syncthreads();
}

__device__ __forceinline__ void write_partials(double* __restrict__ part, double a, double b) {
  block_sum2(a, b);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = a;
    part[NB + blockIdx.x] = b;
  }
}

__device__ __forceinline__ double dot3(const double4_32a& a, const double4_32a& b) {
  return a.x * b.x + a.y * b.y + a.z * b.z;
}

__global__ void k_mu_from_e0(int n, const double4_32a* __restrict__ e0, const double2* __restrict__ al,
                             double4_32a* __restrict__ mu) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
    const double a = al[s].x;
    const double4_32a e = e0[s];
    mu[s] = make_double4_32a(a * e.x, a * e.y, a * e.z, 0.0);
  }
}

// v = hi + lo with hi = fl32(v), lo = fl32(v - hi) (lo skipped when null),
// with lo also (hi, lo) side by side in hl[2 s], hl[2 s + 1]; returns max |hi
// component| for the block maxima of the split vector.
__device__ __forceinline__ float split_store(const double4_32a& v, float4* __restrict__ hi, float4* __restrict__ lo,
                                             float4* __restrict__ hl, int s) {
  if (!hi) return 0.f;
  const float4 h = make_float4(__double2float_rn(v.x), __double2float_rn(v.y), __double2float_rn(v.z), 0.f);
  hi[s] = h;
  if (lo) {
    const float4 l = make_float4(__double2float_rn(v.x - (double)h.x), __double2float_rn(v.y - (double)h.y),
                                 __double2float_rn(v.z - (double)h.z), 0.f);
    lo[s] = l;
    hl[2 * (long long)s] = h;
    hl[2 * (long long)s + 1] = l;
  }
  return fmaxf(fabsf(h.x), fmaxf(fabsf(h.y), fabsf(h.z)));
}

// Max of m over the whole grid into vmax[NB] (the float64 path's reciprocal
// spreading scales its fixed-point grid by it): every block stores its max in
// vmax[blockIdx.x]; the last block to arrive (counter in vmax[NB + 1], back to
// zero afterwards) reduces them. Called by every block of the launch.
__device__ __forceinline__ void write_max_partial(float* __restrict__ vmax, float m) {
  __shared__ float sm[NT / 32];
  __shared__ bool last;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float r = sm[0];
    for (int w = 1; w < NT / 32; ++w) r = fmaxf(r, sm[w]);
    vmax[blockIdx.x] = r;
    __threadfence();
    unsigned* count = reinterpret_cast<unsigned*>(vmax + NB + 1);
    last = atomicAdd(count, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x < 32) {
    __threadfence();
    float r = 0.f;
    for (int k = threadIdx.x; k < (int)gridDim.x; k += 32) r = fmaxf(r, __ldcg(vmax + k));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r = fmaxf(r, __shfl_xor_sync(0xffffffffu, r, o));
    if (threadIdx.x == 0) {
      vmax[NB] = r;
      *reinterpret_cast<unsigned*>(vmax + NB + 1) = 0u;
    }
  }
}

__device__ __forceinline__ double4_32a sum_t(const double4_32a* __restrict__ t, const double4_32a* __restrict__ t2,
                                             int s) {
  double4_32a a = t[s];
  if (t2) {
    const double4_32a b = t2[s];
    a.x += b.x;
    a.y += b.y;
    a.z += b.z;
  }
  return a;
}

// Called once by every block after it stored its partials; true in the block
// that arrived last (every partial is then visible to it). The counter goes
// back to zero for the next launch.
__device__ __forceinline__ bool last_block(int* fl) {
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    unsigned* count = reinterpret_cast<unsigned*>(fl + F_COUNT);
    last = atomicAdd(count, 1u) == gridDim.x - 1;
    if (last) *count = 0u;
  }
  __syncthreads();
  if (last) __threadfence();
  return last;
}

// Block partials of z.z (into part[2 NB + block]) and of max |z32| (into
// vmax[block]); the last block reduces both. Returns true in that block, with
// rms (Debye) in its thread 0, which runs the convergence test.
__device__ __forceinline__ bool finish_z(int n, double zz, float vm, double* __restrict__ part,
                                         float* __restrict__ vmax, int* __restrict__ fl, double& rms) {
  double unused = 0.0;
  block_sum2(zz, unused);
  __shared__ float sm[NT / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) vm = fmaxf(vm, __shfl_xor_sync(0xffffffffu, vm, o));
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = vm;
  __syncthreads();
  if (threadIdx.x == 0) {
    float m = sm[0];
    for (int w = 1; w < NT / 32; ++w) m = fmaxf(m, sm[w]);
    part[2 * NB + blockIdx.x] = zz;
    vmax[blockIdx.x] = m;
  }
  if (!last_block(fl)) return false;
  if (threadIdx.x < 32) {
    double tot = 0.0;
    float m = 0.f;
    for (int k = threadIdx.x; k < (int)gridDim.x; k += 32) {
      tot += __ldcg(part + 2 * NB + k);
      m = fmaxf(m, __ldcg(vmax + k));
    }
    tot = warp_sum(tot);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) {
      vmax[NB] = m;
      rms = kDebye * sqrt(tot / (double)(n > 0 ? n : 1));
    }
  }
  return true;
}

// The solver state for the host: flags [0, 4) and scalars [0, 4) into the
// mapped host readback, by the thread that wrote them last (the host reads
// them after synchronising the stream).
__device__ __forceinline__ void publish(const int* fl, const double* scal, int* __restrict__ hfl,
                                        double* __restrict__ hsc) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    hfl[k] = fl[k];
    hsc[k] = scal[k];
  }
}

// r = E0 - mu/alpha + t (t (+ t2) = T mu); z = alpha r and its float split
// (z32, zlo: the operator's input); convergence test on z. Starts (or
// restarts) the recurrence: the next step has beta = 0.
__global__ void __launch_bounds__(NT) k_cg_init(int n, const double4_32a* __restrict__ e0,
                                                const double4_32a* __restrict__ mu, const double4_32a* __restrict__ t,
                                                const double4_32a* __restrict__ t2, const double2* __restrict__ al,
                                                double4_32a* __restrict__ r, double4_32a* __restrict__ z,
                                                float4* __restrict__ z32, float4* __restrict__ zlo,
                                                float4* __restrict__ zhl, double* __restrict__ part,
                                                float* __restrict__ vmax, double* __restrict__ scal,
                                                int* __restrict__ fl, int* __restrict__ hfl,
                                                double* __restrict__ hsc, double tol) {
  double zz = 0.0;
  float vm = 0.f;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
    const double2 a = al[s];
    const double4_32a e = e0[s], m = mu[s], tt = sum_t(t, t2, s);
    const double4_32a rr = make_double4_32a(e.x - m.x * a.y + tt.x, e.y - m.y * a.y + tt.y, e.z - m.z * a.y + tt.z, 0.0);
    const double4_32a zv = make_double4_32a(a.x * rr.x, a.x * rr.y, a.x * rr.z, 0.0);
    r[s] = rr;
    z[s] = zv;
    vm = fmaxf(vm, split_store(zv, z32, zlo, zhl, s));
    zz += dot3(zv, zv);
  }
  double rms = 0.0;
  if (finish_z(n, zz, vm, part, vmax, fl, rms) && threadIdx.x == 0) {
    scal[2] = rms;
    fl[F_FIRST] = 1;
    const bool conv = rms < tol;
    fl[F_STOP] = conv ? 1 : 0;
    fl[F_STATUS] = conv ? 1 : 0;
    publish(fl, scal, hfl, hsc);
  }
}

// After w's operator part t (+ t2) = T z: w = z/alpha - t; partials r.z, z.w.
__global__ void __launch_bounds__(NT) k_cg_dots(int n, const double4_32a* __restrict__ r,
                                                const double4_32a* __restrict__ z, const double4_32a* __restrict__ t,
                                                const double4_32a* __restrict__ t2, const double2* __restrict__ al,
                                                double4_32a* __restrict__ w, double* __restrict__ part,
                                                const int* __restrict__ fl) {
  pdl_wait();  // first: a kernel never completes before the one it depends on
  if (fl[F_STOP]) return;
  pdl_trigger();
  double rz = 0.0, zw = 0.0;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
    const double ia = al[s].y;
    const double4_32a zv = z[s], tt = sum_t(t, t2, s);
    const double4_32a wv = make_double4_32a(zv.x * ia - tt.x, zv.y * ia - tt.y, zv.z * ia - tt.z, 0.0);
    w[s] = wv;
    rz += dot3(r[s], zv);
    zw += dot3(zv, wv);
  }
  write_partials(part, rz, zw);
}

// One step: scalars from the partials of k_cg_dots, the vector update, the
// new z (and its split), and the convergence / iteration-limit test.
__global__ void __launch_bounds__(NT) k_cg_step(int n, double4_32a* __restrict__ mu, double4_32a* __restrict__ r,
                                                double4_32a* __restrict__ z, double4_32a* __restrict__ p,
                                                double4_32a* __restrict__ q, const double4_32a* __restrict__ w,
                                                const double2* __restrict__ al, float4* __restrict__ z32,
                                                float4* __restrict__ zlo, float4* __restrict__ zhl,
                                                double* __restrict__ part,
                                                float* __restrict__ vmax, double* __restrict__ scal,
                                                int* __restrict__ fl, int* __restrict__ hfl,
                                                double* __restrict__ hsc, double tol, int max_iter,
                                                bool last_of_chunk) {
  pdl_wait();  // first: a kernel never completes before the one it depends on
  if (fl[F_STOP]) return;
  pdl_trigger();
  double rho, m;
  reduce_partials(part, vec_blocks(n), rho, m);
  __shared__ double sbeta, sgamma;
  __shared__ bool bad;
  if (threadIdx.x == 0) {
    double beta = 0.0, den = m;
    if (!fl[F_FIRST]) {
      beta = rho / scal[0];
      den = m - beta * rho / scal[1];
    }
    bad = !(den > 0.0);  // p.Ap <= 0: the operator is not positive definite
    sbeta = beta;
    sgamma = rho / den;
  }
  __syncthreads();
  const double beta = sbeta, gamma = sgamma;
  double zz = 0.0;
  float vm = 0.f;
  if (!bad) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
      const double a = al[s].x;
      const double4_32a zv = z[s], wv = w[s];
      double4_32a pp = p[s], qq = q[s], x = mu[s], rr = r[s];
      pp = make_double4_32a(zv.x + beta * pp.x, zv.y + beta * pp.y, zv.z + beta * pp.z, 0.0);
      qq = make_double4_32a(wv.x + beta * qq.x, wv.y + beta * qq.y, wv.z + beta * qq.z, 0.0);
      x = make_double4_32a(x.x + gamma * pp.x, x.y + gamma * pp.y, x.z + gamma * pp.z, 0.0);
      rr = make_double4_32a(rr.x - gamma * qq.x, rr.y - gamma * qq.y, rr.z - gamma * qq.z, 0.0);
      const double4_32a zn = make_double4_32a(a * rr.x, a * rr.y, a * rr.z, 0.0);
      p[s] = pp;
      q[s] = qq;
      mu[s] = x;
      r[s] = rr;
      z[s] = zn;
      vm = fmaxf(vm, split_store(zn, z32, zlo, zhl, s));
      zz += dot3(zn, zn);
    }
  }
  double rms = 0.0;
  if (finish_z(n, zz, vm, part, vmax, fl, rms) && threadIdx.x == 0) {
    const int it = fl[F_ITERS] + 1;
    fl[F_ITERS] = it;
    fl[F_FIRST] = 0;
    if (bad) {
      fl[F_STOP] = 1;
      fl[F_STATUS] = 3;
      publish(fl, scal, hfl, hsc);
      return;
    }
    scal[0] = rho;
    scal[1] = gamma;
    scal[2] = rms;
    if (rms < tol) {
      fl[F_STOP] = 1;
      fl[F_STATUS] = 1;
    } else if (it >= max_iter) {
      fl[F_STOP] = 1;
      fl[F_STATUS] = 2;
    }
    if (last_of_chunk || fl[F_STOP]) publish(fl, scal, hfl, hsc);
  }
}

__global__ void k_to_sorted(int n, const int* __restrict__ perm, const double* __restrict__ src,
                            double4_32a* __restrict__ dst) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int i = perm[s];
  dst[s] = make_double4_32a(src[3 * i], src[3 * i + 1], src[3 * i + 2], 0.0);
}

__global__ void k_from_sorted(int n, const int* __restrict__ perm, const double4_32a* __restrict__ src,
                              double* __restrict__ dst) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int i = perm[s];
  const double4_32a v = src[s];
  dst[3 * i] = v.x;
  dst[3 * i + 1] = v.y;
  dst[3 * i + 2] = v.z;
}

// a += b in cell order, and dst (caller order) = the sum
__global__ void k_add_from_sorted(int n, const int* __restrict__ perm, double4_32a* __restrict__ a,
                                  const double4_32a* __restrict__ b, double* __restrict__ dst) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int i = perm[s];
  const double4_32a u = a[s], w = b[s];
  const double4_32a v = make_double4_32a(u.x + w.x, u.y + w.y, u.z + w.z, 0.0);
  a[s] = v;
  dst[3 * i] = v.x;
  dst[3 * i + 1] = v.y;
  dst[3 * i + 2] = v.z;
}

__global__ void __launch_bounds__(NT) k_split(int n, const double4_32a* __restrict__ v, float4* __restrict__ hi,
                                             float4* __restrict__ lo, float4* __restrict__ hl,
                                             float* __restrict__ vmax) {
  float vm = 0.f;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x)
    vm = fmaxf(vm, split_store(v[s], hi, lo, hl, s));
  write_max_partial(vmax, vm);
}

// U = -1/2 C sum mu . E0 over the caller's [N][3] arrays
__global__ void __launch_bounds__(NT) k_energy_partial(long long m, const double* __restrict__ mu,
                                                       const double* __restrict__ e0, double* __restrict__ part) {
  double s = 0.0;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < m; k += (long long)gridDim.x * blockDim.x)
    s += mu[k] * e0[k];
  write_partials(part, s, 0.0);
}

__global__ void __launch_bounds__(NT) k_energy_finish(const double* __restrict__ part, double* __restrict__ out,
                                                      double* __restrict__ hout) {
  double s, unused;
  reduce_partials(part, NB, s, unused);
  if (threadIdx.x == 0) {
    *out = -0.5 * kCoulomb * s;
    *hout = *out;
  }
}

}  // namespace

void launch_to_sorted(amp_ctx* c, const double* src, double4_32a* dst) {
  c->n_launch += 1;
  k_to_sorted<<<amp_blocks(c->n, 256), 256, 0, c->stream>>>(c->n, c->perm, src, dst);
}

void launch_from_sorted(amp_ctx* c, const double4_32a* src, double* dst) {
  c->n_launch += 1;
  k_from_sorted<<<amp_blocks(c->n, 256), 256, 0, c->stream>>>(c->n, c->perm, src, dst);
}

void launch_add_from_sorted(amp_ctx* c, double4_32a* a, const double4_32a* b, double* dst) {
  c->n_launch += 1;
  k_add_from_sorted<<<amp_blocks(c->n, 256), 256, 0, c->stream>>>(c->n, c->perm, a, b, dst);
}

void launch_to32(amp_ctx* c, const double4_32a* v, float4* o) {
  c->n_launch += 1;
  k_split<<<vec_blocks(c->n), NT, 0, c->stream>>>(c->n, v, o, nullptr, nullptr, c->vmax_part);
}

void launch_split(amp_ctx* c, const double4_32a* v, float4* hi, float4* lo) {
  c->n_launch += 1;
  k_split<<<vec_blocks(c->n), NT, 0, c->stream>>>(c->n, v, hi, lo, lo ? c->vhl : nullptr, c->vmax_part);
}

// Real-space kernel of an operator application.
enum RealMode { kRealDf, kRealF32, kRealDirectDf };

// T v = t (+ t2). With t2 == nullptr the whole product lands in t. With t2
// given (periodic systems) the reciprocal part runs on the side stream into t2
// while the real-space kernel runs on the main stream into t: the two parts
// are independent. The real-space kernel starts once the dipoles are spread:
// the spreading keeps every SM busy by itself, while the three FFT passes
// that follow are latency bound and leave most of the GPU to the real-space
// kernel. The main stream waits for the side stream before returning. The
// reciprocal part is the double-float chain for the float64 path and the
// mixed path's float64 check (kRealDirectDf, which first splits v into
// (p32, plo) for both parts), the float32 chain for the mixed operator.
// Whether the real-space kernel waits for the reciprocal chain's spreading
// (it then shares the GPU with the latency-bound FFT passes rather than with
// the spreading, which fills every SM) or starts at the fork. The chain's
// kernels are launched early (programmatic dependent launch) and hold their
// SM resources while they wait for the kernel before them; on large grids
// these are many cluster CTAs, and a real-space kernel that starts after the
// spreading finds the SMs taken. Measured (float64 path): water-23556
// (K = 64) solve 0.873 ms after the spreading, 1.011 ms from the fork;
// water-96000 (K = 100) 4.01 ms after the spreading, 2.87 ms from the fork.
// The mixed operator's chain on large grids is cuFFT's, launched the
// ordinary way: after the spreading at both sizes (1.94 vs 2.17 ms at
// water-96000). The float64 residual check starts it at the fork.
static bool real_after_spread(const amp_ctx* c, RealMode mode) {
  if (mode == kRealDirectDf) return false;
  if (mode == kRealDf) return c->n < kTRealForkAtoms;
  return true;
}

static int fork_join_T(amp_ctx* c, const double4_32a* v, const float4* v32, const float4* vlo, double4_32a* t,
                       double4_32a* t2, RealMode mode) {
  int r;
  if (mode == kRealDirectDf) {
    launch_split(c, v, c->p32, c->plo);
    v32 = c->p32;
    vlo = c->plo;
  }
  if (t2) {
    cudaEventRecord(c->ev_fork, c->stream);
    cudaStreamWaitEvent(c->side, c->ev_fork, 0);
    {
      PhaseScope ps(c, AMP_PHASE_T_RECIP, c->side);
      c->spread_event = real_after_spread(c, mode);
      r = mode == kRealF32 ? pme_dipole_field32(c, v32, t2, c->side, true)
                           : pme_dipole_field(c, v, v32, vlo, t2, c->side, true);
      if (c->spread_event) cudaStreamWaitEvent(c->stream, c->ev_spread, 0);
      c->spread_event = false;
    }
    cudaEventRecord(c->ev_join, c->side);
    if (r) {
      cudaStreamWaitEvent(c->stream, c->ev_join, 0);
      return r;
    }
  }
  {
    PhaseScope ps(c, AMP_PHASE_T_REAL);
    if (mode == kRealDirectDf)
      launch_t_real_fp64_direct(c, v, t);
    else if (mode == kRealDf)
      launch_t_real(c, v, t);
    else
      launch_t_real32(c, v32, v, t);
  }
  if (t2) {
    cudaStreamWaitEvent(c->stream, c->ev_join, 0);
    return AMP_OK;
  }
  PhaseScope ps(c, AMP_PHASE_T_RECIP);
  if (mode == kRealF32) return pme_dipole_field32(c, v32, t, c->stream, false);
  return pme_dipole_field(c, v, v32, vlo, t, c->stream, false);
}

// t (+ t2) = T v in the solver's working precision. v32 (+ vlo) must mirror
// v: mixed, v32 = fl32(v); float64, v = v32 + vlo (double-float split).
int apply_T_sorted(amp_ctx* c, const double4_32a* v, const float4* v32, const float4* vlo, double4_32a* t,
                   double4_32a* t2) {
  const bool fp64 = c->cfg.precision == AMP_FP64;
  if (c->cluster) {
    PhaseScope ps(c, AMP_PHASE_T_REAL);
    cluster_t(c, v, v32, t, fp64);
    if (t2) cudaMemsetAsync(t2, 0, sizeof(double4_32a) * c->n, c->stream);
    return AMP_OK;
  }
  return fork_join_T(c, v, v32, vlo, t, t2, fp64 ? kRealDf : kRealF32);
}

// Mixed path: t (+ t2) = T v with every term in float64 (pair tensors recomputed).
static int apply_T_sorted_fp64_check(amp_ctx* c, const double4_32a* v, double4_32a* t, double4_32a* t2) {
  PhaseScope ps(c, AMP_PHASE_FP64_CHECK);
  if (c->cluster) {
    cluster_t(c, v, nullptr, t, true);
    if (t2) cudaMemsetAsync(t2, 0, sizeof(double4_32a) * c->n, c->stream);
    return AMP_OK;
  }
  return fork_join_T(c, v, nullptr, nullptr, t, t2, kRealDirectDf);
}

// The last k_cg_init / k_cg_step that ran wrote the flags and scalars into
// the mapped host readback (hibuf[0, 4), hbuf[0, 4)): synchronise and read.
static int read_flags(amp_ctx* c) { return cuda_check(c, cudaStreamSynchronize(c->stream), "solver flag read"); }

// One iteration: w's operator part T z (skipped on the device once the solve
// has stopped), then k_cg_dots and k_cg_step. The host reads the flags after
// the last iteration of a chunk: that step, or the one that stops the solve,
// publishes them (a write to host memory at the end of every step would
// lengthen each step's completion).
static int enqueue_iteration(amp_ctx* c, bool last_of_chunk) {
  const int n = c->n;
  cudaStream_t st = c->stream;
  float4* lo = c->cfg.precision == AMP_MIXED ? nullptr : c->plo;
  c->op_stop = c->iflags + F_STOP;
  int r = apply_T_sorted(c, c->zv, c->p32, lo, c->tv, c->trec);
  c->op_stop = nullptr;
  if (r) return r;
  PhaseScope ps(c, AMP_PHASE_PCG);
  c->n_launch += 2;
  const int nb = vec_blocks(n);
  launch_pdl(k_cg_dots, dim3(nb), dim3(NT), 0, st, n, c->res, c->zv, c->tv, c->trec, c->alph, c->wv, c->partials,
             c->iflags);
  launch_pdl(k_cg_step, dim3(nb), dim3(NT), 0, st, n, c->mu, c->res, c->zv, c->pv, c->qv, c->wv, c->alph, c->p32,
             lo, lo ? c->vhl : nullptr, c->partials, c->vmax_part, c->scal, c->iflags, c->hibuf_d, c->hbuf_d,
             c->cfg.tol_debye, c->cfg.max_iter, last_of_chunk);
  return AMP_OK;
}

// Residual of the current mu with the float64 or working operator, then
// restart the recurrence from it.
static int restart(amp_ctx* c, bool fp64_operator) {
  const bool mixed = c->cfg.precision == AMP_MIXED;
  float4* lo = mixed ? nullptr : c->plo;
  int r;
  if (fp64_operator && mixed) {
    r = apply_T_sorted_fp64_check(c, c->mu, c->tv, c->trec);
  } else {
    // the float split of mu goes through the operator-input buffers, which k_cg_init rewrites
    launch_split(c, c->mu, c->p32, lo);
    r = apply_T_sorted(c, c->mu, c->p32, lo, c->tv, c->trec);
  }
  if (r) return r;
  PhaseScope ps(c, AMP_PHASE_PCG);
  c->n_launch += 1;
  k_cg_init<<<vec_blocks(c->n), NT, 0, c->stream>>>(c->n, c->E0s, c->mu, c->tv, c->trec, c->alph, c->res, c->zv, c->p32, lo,
                                      lo ? c->vhl : nullptr, c->partials, c->vmax_part, c->scal, c->iflags,
                                      c->hibuf_d, c->hbuf_d, c->cfg.tol_debye);
  return AMP_OK;
}

// ASPC predictor (Kolafa, J. Comput. Chem. 25, 335 (2004)): the initial
// dipoles of a solve along a trajectory from the last k + 2 converged ones,
//   mu_0 = sum_{j=1}^{k+2} B_j mu_{-j},
//   B_j = (-1)^{j+1} j C(2k+4, k+2-j) / C(2k+2, k+1)
// (k = 0: 2 mu_{-1} - mu_{-2}; k = 1: 2.5 mu_{-1} - 2 mu_{-2} + 0.5 mu_{-3}).
constexpr int kMaxHistory = 8;
struct Predictor {
  int nh;
  const double4_32a* v[kMaxHistory];
  double b[kMaxHistory];
};

__global__ void k_predict(int n, Predictor P, double4_32a* __restrict__ mu) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  double x = 0.0, y = 0.0, z = 0.0;
  for (int t = 0; t < P.nh; ++t) {
    const double4_32a h = P.v[t][s];
    x += P.b[t] * h.x;
    y += P.b[t] * h.y;
    z += P.b[t] * h.z;
  }
  mu[s] = make_double4_32a(x, y, z, 0.0);
}

static double binom(int a, int b) {
  if (b < 0 || b > a) return 0.0;
  double r = 1.0;
  for (int i = 1; i <= b; ++i) r = r * (double)(a - b + i) / (double)i;
  return r;
}

bool predict_guess(amp_ctx* c) {
  const int k = c->pred_order, m = k + 2;
  if (k < 0 || c->hist_len < m) return false;
  Predictor P{};
  P.nh = m;
  amp_predictor_coefficients(k, P.b);
  const int cap = (int)(c->hist_cap / (c->n > 0 ? c->n : 1));
  for (int j = 1; j <= m; ++j) {  // j-th most recent
    const int slot = ((c->hist_head - j) % cap + cap) % cap;
    P.v[j - 1] = c->hist + (long long)slot * c->n;
  }
  c->n_launch += 1;
  k_predict<<<amp_blocks(c->n, 256), 256, 0, c->stream>>>(c->n, P, c->mu);
  return true;
}

int push_history(amp_ctx* c) {
  const int k = c->pred_order;
  if (k < 0) return AMP_OK;
  const int m = k + 2;
  if ((long long)m * c->n > c->hist_cap) {
    dev_free(c, c->hist);
    c->hist = nullptr;
    c->hist_cap = 0;
    int r;
    if ((r = dev_alloc(c, &c->hist, (long long)m * c->n))) return r;
    c->hist_cap = (long long)m * c->n;
    c->hist_len = c->hist_head = 0;
  }
  const int cap = (int)(c->hist_cap / c->n);
  c->hist_head %= cap;
  cudaMemcpyAsync(c->hist + (long long)c->hist_head * c->n, c->mu, sizeof(double4_32a) * c->n,
                  cudaMemcpyDeviceToDevice, c->stream);
  c->hist_head = (c->hist_head + 1) % cap;
  if (c->hist_len < m) ++c->hist_len;
  return AMP_OK;
}

int solve(amp_ctx* c, bool use_guess) {
  const bool mixed = c->cfg.precision == AMP_MIXED;
  cudaStream_t st = c->stream;
  int r;
  if (!use_guess) c->n_launch += 1;
  if (!use_guess) k_mu_from_e0<<<vec_blocks(c->n), NT, 0, st>>>(c->n, c->E0s, c->alph, c->mu);
  if ((r = cuda_check(c, cudaMemsetAsync(c->iflags, 0, sizeof(int) * 5, st), "memset"))) return r;
  if ((r = restart(c, !mixed))) return r;
  // Iterations are enqueued in chunks between reads of the device flags; a
  // read is a host round trip (~30 us on GB300, with the GPU idle). The first
  // chunk is the iteration count that the previous solve on this context
  // needed, so that a run of similar solves reads the flags once; later
  // chunks are kPcgChunk. Iterations enqueued after convergence cost only
  // their launches (every kernel returns at once on the stop flag).
  int chunk = c->last_iters > 0 ? c->last_iters : kPcgChunk;
  c->stats.fp64_checks = 0;
  for (int round = 0; round < 8; ++round) {
    while (true) {
      for (int k = 0; k < chunk; ++k)
        if ((r = enqueue_iteration(c, k == chunk - 1))) return r;
      if ((r = read_flags(c))) return r;
      chunk = kPcgChunk;
      if (c->hibuf[F_STOP]) break;
    }
    if (round == 0) c->last_iters = std::max(1, std::min(c->hibuf[F_ITERS], c->cfg.max_iter));
    if (!mixed || c->hibuf[F_STATUS] != 1) break;
    // mixed: check the converged dipoles with the float64 operator
    if ((r = restart(c, true))) return r;
    c->stats.fp64_checks++;
    if ((r = read_flags(c))) return r;
    if (c->hibuf[F_STATUS] == 1 || c->hibuf[F_ITERS] >= c->cfg.max_iter) break;
  }
  if ((r = cuda_check(c, cudaGetLastError(), "solver launch"))) return r;
  c->stats.iters = c->hibuf[F_ITERS];
  c->stats.rms = c->hbuf[2];
  const int status = c->hibuf[F_STATUS];
  if (status == 3) return fail(c, AMP_ERR_NOT_CONVERGED, "PCG breakdown: p.Ap <= 0");
  if (status != 1)
    return fail(c, AMP_ERR_NOT_CONVERGED, "PCG not converged after %d iterations (RMS %.3e D)", c->stats.iters,
                c->stats.rms);
  return AMP_OK;
}

int energy(amp_ctx* c, const double* mu, const double* E0, double* U) {
  {
    PhaseScope ps(c, AMP_PHASE_ENERGY);
    c->n_launch += 2;
    k_energy_partial<<<NB, NT, 0, c->stream>>>(3LL * c->n, mu, E0, c->partials);
    k_energy_finish<<<1, NT, 0, c->stream>>>(c->partials, c->scal + 3, c->hbuf_d + 3);
  }
  int r = cuda_check(c, cudaStreamSynchronize(c->stream), "energy");
  if (r) return r;
  *U = c->hbuf[3];
  return AMP_OK;
}

}  // namespace amp

extern "C" int amp_predictor_coefficients(int order, double* b) {
  if (order < 0 || order > 6 || !b) return AMP_ERR_ARG;
  const int k = order;
  for (int j = 1; j <= k + 2; ++j)
    b[j - 1] = ((j + 1) % 2 == 0 ? 1.0 : -1.0) * j * amp::binom(2 * k + 4, k + 2 - j) / amp::binom(2 * k + 2, k + 1);
  return AMP_OK;
}
