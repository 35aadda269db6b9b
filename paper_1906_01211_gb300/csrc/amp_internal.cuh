// Internal declarations shared by the translation units of libamoebapol.
//
// Data layout on the device (all arrays are in "cell order": atoms re-ordered
// so that the atoms of one cell are contiguous; perm[s] is the caller's index
// of sorted atom s):
//   atomA[s] = (x, y, z, q)                 float64, unwrapped positions
//   atomB[s] = (dx, dy, dz, 1/sqrt(alpha))  permanent dipole
//   atomC[s] = (Qxx, Qyy, Qzz, Qxy)
//   atomD[s] = (Qxz, Qyz, thole, mol)       mol stored as a double
//   pos32[s] = positions wrapped into [0, L), float32 (list pre-filter, mixed)
//   vectors (E0, mu, residual, ...) are double4_32a (x, y, z, 0) per atom.
// Neighbour lists:
//   full list  CSR rows full_start[s]..full_start[s+1]: entry k holds the
//              neighbour index full_j[k] and full_ref[k] = 2*pid + side, where
//              pid is the unique-pair id and side = 0 if the row owns the pair;
//              a row lists its owned pairs first, then the others by pair id;
//   half list  (half_i[pid], half_j[pid]) for every unique pair, owned by the
//              row for which (i < j) != ((i + j) odd) — each pair exactly once,
//              about half of each row's neighbours.
// Pair data indexed by pid (computed once per geometry):
//   T32: the mixed path's float32 tensor once per full-list entry, in entry
//     order: (xx, yy, zz, xy) as float4 from the start, (xz, yz) as float2
//     after cap_full entries
//   C64: the float64 path's pair tensor T = -b1 I + b2 r r^T as its two
//     scalars, once per full-list entry in entry order: (b1 hi, b1 lo,
//     b2 hi, b2 lo), 16 bytes; the product kernel rebuilds r from xhl
//   Ep64/Ep32[pid*6 + side*3 + a]         permanent field at the side's atom
#pragma once

#include <cuda_runtime.h>
#include <cufft.h>

#include <cstddef>
#include <cstdint>
#include <vector>

#include "amoebapol.h"

namespace amp {

constexpr int kOrder = 5;
constexpr double kDebye = 4.8032047;
constexpr double kCoulomb = 332.0637133;
constexpr double kSqrtPi = 1.7724538509055160273;
constexpr int kRowGroup = 16;       // lanes that share one neighbour row
constexpr int kTRealForkAtoms = 48000;  // float64 path: the real-space kernel starts at the fork from here on
constexpr int kForcePairStride = 24;  // backward per-pair record (doubles)
constexpr int kForceAtomStride = 16;  // backward per-atom reciprocal record (doubles)
constexpr int kReduceBlocks = 296;  // 2 x 152 SMs: blocks of the PCG kernels
constexpr int kReduceThreads = 256;

struct Stats {
  int iters = 0;
  double rms = 0.0;
  int fp64_checks = 0;
};

}  // namespace amp

struct amp_ctx {
  amp_config cfg{};
  cudaStream_t stream = nullptr;
  char err[512] = {0};
  int n = 0, n_cap = 0;

  // cells
  int nc = 0, ncell = 0, ncell_cap = 0;
  int *cell_of = nullptr, *cell_count = nullptr, *cell_start = nullptr, *cell_fill = nullptr;
  int *perm = nullptr, *inv_perm = nullptr, *slot_tmp = nullptr;
  double4_32a *atomA = nullptr, *atomB = nullptr, *atomC = nullptr, *atomD = nullptr;
  double2* alph = nullptr;  // (alpha, 1/alpha) per sorted atom
  float4* mp_df = nullptr;  // float64 path: q, d, Theta as hi/lo float pairs, 5 float4 per atom
  // float64 path, per atom: (x, y, z, 1/sqrt(alpha)) hi, the same lo, (thole hi, lo, molecule, 0)
  float4* pd = nullptr;
  float4* xhl = nullptr;    // float64 path, per atom: (x, y, z, 0) hi, the same lo (32 bytes)
  float2* dfm = nullptr;    // float64 path: table of the double-float elementary functions
  float4* pos32 = nullptr;

  // neighbour lists
  int *full_cnt = nullptr, *half_cnt = nullptr, *full_start = nullptr, *half_start = nullptr;
  int *full_j = nullptr, *full_ref = nullptr, *half_i = nullptr, *half_j = nullptr, *tr_tmp = nullptr;
  int* pos_tr = nullptr;  // full-list position of each pair's entry in its non-owner's row
  int* intra = nullptr;   // float64 path: [0] count, then the pair ids of two sites of one molecule
  // list reuse: skin for the next build; the candidates (pairs within cutoff
  // + skin_built at the last cell search, CSR) and the sorted positions then
  double skin = 0.0, skin_built = 0.0;
  int *cand_start = nullptr, *cand_j = nullptr;
  long long cand_cap = 0, cand_start_cap = 0;
  double4_32a* xref = nullptr;
  double4_32a* abak = nullptr;  // positions before an update (put back if it is refused)
  float4* pbak = nullptr;
  long long n_full = 0, n_half = 0, cap_full = 0, cap_half = 0;
  int* flags = nullptr;  // [0] bit 1 list transpose failure, bit 2 bad alpha, bit 4 slab overflow
  int* slab = nullptr;   // single-pass list: owned neighbours per atom, fixed row capacity
  long long slab_cap = 0;

  // pair data
  float4* C64 = nullptr;
  double* Ep64 = nullptr;
  float* T32 = nullptr;
  float* Ep32 = nullptr;

  // PME
  int K = 0;
  double* theta = nullptr;  // [n][3 axes][4 derivatives][5 points]
  float* theta32 = nullptr;
  float2* theta_df = nullptr;  // weights and first derivatives as hi/lo [n][3][2][5] (dipole products)
  bool theta64_valid = false;   // theta (float64) matches the current system (built on first use)
  float2* phi_df = nullptr;    // float64 path: grid potential as hi/lo pairs for the gather
  // float64 path's dipole spreading: 64-bit fixed-point grid (integer
  // atomics, exact and order-independent), scaled by 2^fx_info[0]; fx_info[1]
  // bounds the atoms that reach one grid point; kcount = atoms per base cell.
  unsigned long long* gridfx = nullptr;
  int* fx_info = nullptr;  // [0] scale exponent of the last spread, [1] atoms per base cell (max)
  int* kcount = nullptr;
  // max |hi component| of the last split vector: [0, kReduceBlocks) per block,
  // [kReduceBlocks] the whole vector, [kReduceBlocks + 1] arrival counter
  float* vmax_part = nullptr;
  float4* fft_grid = nullptr;  // double-float complex half spectrum of the own FFT (its grids)
  float2* fft_G = nullptr;     // influence function on that half spectrum, hi/lo
  float4* fft_tw = nullptr;    // twiddles (cos hi, lo, sin hi, lo)
  // mixed path's float32 reciprocal chain: spreading grid (kept at zero
  // between applications), grid potential, and the own FFT's float32 half
  // spectrum and twiddles (G: G32)
  float* spread32 = nullptr;
  float* phi32 = nullptr;
  float2* fft_grid32 = nullptr;
  float2* fft_tw32 = nullptr;
  // the own FFT's float64 variant (the permanent field): half spectrum,
  // twiddles; phi64 its output grid potential (G: G64)
  double2* fft_grid64 = nullptr;
  double2* fft_tw64 = nullptr;
  double* spread64 = nullptr;  // the permanent multipoles' float64 grid (kept zero between uses)
  double* phi64 = nullptr;
  int4* gbase = nullptr;    // [n] base grid index per axis
  double* grid64 = nullptr;
  double2* cgrid64 = nullptr;
  double* G64 = nullptr;
  double* bmod = nullptr;  // B-spline moduli |b(m)|^2, m = 0 .. K-1
  float* grid32 = nullptr;
  float2* cgrid32 = nullptr;
  float* G32 = nullptr;
  cufftHandle plan_d2z = 0, plan_z2d = 0, plan_r2c = 0, plan_c2r = 0;
  bool plans = false;

  // vectors in cell order
  double4_32a *E0s = nullptr, *mu = nullptr, *res = nullptr, *zv = nullptr, *pv = nullptr;
  double4_32a *qv = nullptr, *tv = nullptr, *tmp = nullptr;
  double4_32a* trec = nullptr;  // reciprocal part of T*v, computed on the side stream
  double4_32a* wv = nullptr;    // the solver's w = A z
  // While the solver enqueues an iteration: its device stop flag, which the
  // operator's kernels test on entry (null: always run).
  const int* op_stop = nullptr;
  cudaStream_t side = nullptr;  // second stream: PME beside the real-space kernel
  int n_sm = 1;                 // streaming multiprocessors of the device
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // recorded on the side stream after the geometry's reciprocal-space work
  // (weights, permanent field's reciprocal part into e0rec); every call that
  // follows amp_set_system / amp_update_positions waits for it once
  cudaEvent_t ev_geom = nullptr;
  bool geom_pending = false;
  double4_32a* e0rec = nullptr;  // reciprocal part of the permanent field (float64, cell order)
  double4_32a* e0intra = nullptr;  // float64 path: the intramolecular (excluded) permanent-field terms
  // recorded after the dipole spreading when spread_event is set: the
  // real-space kernel waits for it, so it runs beside the FFTs only
  cudaEvent_t ev_spread = nullptr;
  bool spread_event = false;
  float4* p32 = nullptr;  // float part of p (mixed: p in float32; float64: hi of hi + lo)
  float4* plo = nullptr;  // float64 path: p - hi, so that hi + lo carries p to ~48 bits
  float4* vhl = nullptr;  // float64 path: (p32[s], plo[s]) side by side, one 32-byte record per atom
  double* partials = nullptr;  // block partial sums (two sets)
  int n_parts_cap = 0;
  double* scal = nullptr;      // device scalars of the solver: rz[2], rms, pq
  int* iflags = nullptr;       // device solver state: stop, iters, conv, status
  // Pinned, mapped host readback. Small results reach it by a copy, or are
  // written by the kernel that finishes them through the device aliases
  // (hbuf_d, hibuf_d): the host reads them after a stream synchronisation,
  // and a copy-engine transfer (~3.4 us per round trip) is saved.
  double* hbuf = nullptr;
  int* hibuf = nullptr;
  double* hbuf_d = nullptr;
  int* hibuf_d = nullptr;

  // phase timers
  bool prof = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<int> ev_phase;  // phase of each begin/end pair in flight
  int ev_used = 0;
  int ev_open = 0;
  double prof_ms[AMP_NPHASE] = {0};
  long long prof_cnt[AMP_NPHASE] = {0};

  // backward buffers (allocated by the first amp_forces call)
  double* force_pair = nullptr;
  long long force_pair_cap = 0;
  double* force_recip = nullptr;
  int force_atom_cap = 0;
  double* grid64b = nullptr;
  float* grid32b = nullptr;
  double* mpole_e = nullptr;  // per-atom permanent-multipole energy (sorted order)
  double4_32a* tcg = nullptr;  // TCG-1 vectors (u, r, z, T z, v, T v, c, P/2, kappa z/2)
  long long tcg_cap = 0;
  double* tcg_sc = nullptr;    // TCG-1 scalars (w, s, t, gamma, w/t, kappa, breakdown, U)
  int mpole_e_cap = 0;

  // isolated cluster (box == 0): all-pairs kernels, column-slice partial sums
  bool cluster = false;
  double4_32a* cluster_part = nullptr;
  float4* clu32 = nullptr;  // mixed clusters: (x, y, z, 1/sqrt(alpha)), (thole, 0, 0, 0) per atom
  int clu32_cap = 0;
  long long cluster_part_cap = 0;

  long long n_launch = 0;      // kernels this library has launched (own kernels only)
  std::vector<void*> allocs;   // every device allocation, freed by amp_destroy
  std::vector<size_t> alloc_sizes;
  long long bytes = 0;         // device bytes the context holds
  amp::Stats stats;
  int last_iters = 0;  // iterations of the last solve (first chunk of the next one)
  // ASPC warm start: order (-1 off), ring of the last order + 2 converged
  // dipole vectors (cell order), cleared by set_system
  int pred_order = -1, hist_len = 0, hist_head = 0;
  double4_32a* hist = nullptr;
  long long hist_cap = 0;  // vectors x atoms allocated
  bool have_system = false;
};

namespace amp {

int fail(amp_ctx* c, int code, const char* fmt, ...);
int dev_alloc_bytes(amp_ctx* c, void** p, size_t bytes);
void dev_free(amp_ctx* c, void* p);
template <typename T>
inline int dev_alloc(amp_ctx* c, T** p, long long count) {
  void* q = nullptr;
  int r = dev_alloc_bytes(c, &q, sizeof(T) * (size_t)(count > 0 ? count : 1));
  *p = (T*)q;
  return r;
}
int cuda_check(amp_ctx* c, cudaError_t e, const char* what);
void ctx_bind_stream(amp_ctx* c, cudaStream_t st);

// Phase timers: record an event pair around a phase on the context stream.
int prof_begin(amp_ctx* c, int phase, cudaStream_t st);
void prof_end(amp_ctx* c, int slot, cudaStream_t st);
int prof_resolve(amp_ctx* c);
struct PhaseScope {
  amp_ctx* c;
  cudaStream_t st;
  int slot;
  PhaseScope(amp_ctx* c_, int ph) : c(c_), st(c_->stream) { slot = prof_begin(c, ph, st); }
  PhaseScope(amp_ctx* c_, int ph, cudaStream_t s) : c(c_), st(s) { slot = prof_begin(c, ph, st); }
  ~PhaseScope() { prof_end(c, slot, st); }
};

// neighbour lists (amp_nblist.cu)
int build_cells_and_lists(amp_ctx* c, const double* xyz, const double* q, const double* dip,
                          const double* quad, const double* alpha, const double* thole,
                          const int* mol);
int filter_lists(amp_ctx* c);  // exact lists from the stored candidates
int reuse_lists(amp_ctx* c, const double* xyz, bool* reused);  // new positions if within skin/2

// pair terms and real-space sums (amp_pair.cu)
void launch_pair_build(amp_ctx* c);
int dfm_setup(amp_ctx* c);  // builds c->dfm
void dfm_host_table(std::vector<float2>& tab);  // the table of c->dfm, on the host
void launch_e0_real(amp_ctx* c, double4_32a* out);  // out = real-space E0 + self
// out = T_real v + self v (float64 path, double-float arithmetic; vhi + vlo = v)
void launch_t_real(amp_ctx* c, const double4_32a* v, double4_32a* out);
void launch_t_real32(amp_ctx* c, const float4* v32, const double4_32a* v64, double4_32a* out);
void launch_t_real_fp64_direct(amp_ctx* c, const double4_32a* v, double4_32a* out);

// PME (amp_pme.cu)
int pme_setup(amp_ctx* c);
int pme_alloc_atoms(amp_ctx* c, int n_cap);
int pme_influence(amp_ctx* c);

// own 3D FFT convolution (amp_fft.cuh): even 2,3,5-smooth grids from 16 to 128 (the list in amp_fft.cuh)
bool fft_own_supported(int K);
int fft_own_setup(amp_ctx* c);  // buffers and twiddles (K only); G comes from pme_influence
constexpr int kOwnF32MaxK = 64;  // the mixed operator's own float32 FFT up to this grid, cuFFT above
void fft_df_convolve(amp_ctx* c, cudaStream_t st);   // gridfx (zeroed on the way) -> phi_df, double-float
void fft_f32_convolve(amp_ctx* c, cudaStream_t st);  // spread32 (zeroed on the way) -> phi32, float32
void fft_f64_convolve(amp_ctx* c, cudaStream_t st, double* grid, double* phi);  // grid (zeroed on the way) -> phi
void launch_pme_theta(amp_ctx* c, cudaStream_t st);
void pme_theta64(amp_ctx* c, cudaStream_t st);  // float64 B-spline weights (permanent field, force kernels)
int pme_geometry(amp_ctx* c);  // weights and e0rec on the side stream (ev_geom)
void join_geometry(amp_ctx* c);  // the context stream waits for pme_geometry's work
// reciprocal field of dipoles on stream st: out += field (set: out = field);
// double-float chain from the split v32 + vlo (vlo null: v32 alone)
int pme_dipole_field(amp_ctx* c, const double4_32a* v, const float4* v32, const float4* vlo, double4_32a* out,
                     cudaStream_t st, bool set);
// the mixed path's operator: the float32 chain from v32
int pme_dipole_field32(amp_ctx* c, const float4* v32, double4_32a* out, cudaStream_t st, bool set);

// solver (amp_pcg.cu)
void launch_to_sorted(amp_ctx* c, const double* src, double4_32a* dst);
void launch_from_sorted(amp_ctx* c, const double4_32a* src, double* dst);
// a += b (cell order), and dst (caller order) = the sum
void launch_add_from_sorted(amp_ctx* c, double4_32a* a, const double4_32a* b, double* dst);
int solve(amp_ctx* c, bool use_guess);
bool predict_guess(amp_ctx* c);  // c->mu from the solution history; false if too short
int push_history(amp_ctx* c);     // c->mu into the solution history
void launch_to32(amp_ctx* c, const double4_32a* v, float4* o);
void launch_split(amp_ctx* c, const double4_32a* v, float4* hi, float4* lo);  // v = hi + lo

// backward (amp_forces.cu)
int forces(amp_ctx* c, const double4_32a* mu_sorted, double* F, double* gq, double* gd, double* gt);
int force_buffers(amp_ctx* c);
// float64 (or float32) grid potential of the dipoles v, or of the permanent
// multipoles (multipoles = true), through cuFFT: the backward kernels' grids
int pme_potential(amp_ctx* c, bool fp32, bool multipoles, const double4_32a* v, const float4* v32, void* grid_out,
                  cudaStream_t st);
int multipole_energy(amp_ctx* c, double* U, double* F, double* gq, double* gd, double* gt);
// gradients of sf c.E + a1.T b1 + a2.T b2 (cell-order vectors), as forces and moment gradients
int bilinear_forces(amp_ctx* c, const double4_32a* cv, double sf, const double4_32a* a1, const double4_32a* b1,
                    const double4_32a* a2, const double4_32a* b2, double* F, double* gq, double* gd, double* gt,
                    const double4_32a* intra_mu, double intra_s);
// the two-field gradients (work: two vectors)
int two_rhs_forces(amp_ctx* c, double s, const double4_32a* mu_d, const double4_32a* mu_p, double4_32a* work,
                   double* F, double* gq, double* gd, double* gt);
// out += the permanent field with intramolecular scale s minus that with scale 0
void launch_intra_scaled(amp_ctx* c, double s, double4_32a* out);
int apply_T_sorted(amp_ctx* c, const double4_32a* v, const float4* v32, const float4* vlo, double4_32a* t,
                   double4_32a* t2);
void launch_split_multipoles(amp_ctx* c);  // pd and mp_df from the atom records
int energy(amp_ctx* c, const double* mu, const double* E0, double* U);

// isolated clusters (amp_cluster.cu)
constexpr int kClusterMaxSlices = 32;
int cluster_setup(amp_ctx* c, const double* xyz, const double* q, const double* dip, const double* quad,
                  const double* alpha, const double* thole, const int* mol);
void cluster_permanent_field(amp_ctx* c, double4_32a* out);
void cluster_t(amp_ctx* c, const double4_32a* v, const float4* v32, double4_32a* out, bool fp64);

}  // namespace amp

namespace amp {

// ---- double-float arithmetic (a value is hi + lo, two floats, |lo| <= ulp(hi)/2)
// Error-free transformations with round-to-nearest intrinsics, which the
// compiler never contracts: two-sum (Knuth) and the FMA two-product give about
// 48 significant bits, enough for float64-level results (1e-14 relative) on a
// GPU whose float32 rate is ~58 times its float64 rate. Conversions between
// float and double run at the float64 rate, so values that are reused are
// split once and kept as hi/lo pairs.
struct dflt {
  float hi, lo;
};

__device__ __forceinline__ dflt df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

__device__ __forceinline__ dflt df_quick(float s, float t) {  // renormalise, |s| >= |t|
  const float h = __fadd_rn(s, t);
  return {h, __fsub_rn(t, __fsub_rn(h, s))};
}

// acc += (ahi + alo) * (bhi + blo)
__device__ __forceinline__ void df_fma(dflt& acc, float ahi, float alo, float bhi, float blo) {
  const float p = __fmul_rn(ahi, bhi);
  float e = __fmaf_rn(ahi, bhi, -p);
  e = __fmaf_rn(ahi, blo, e);
  e = __fmaf_rn(alo, bhi, e);
  const dflt s = df_two_sum(acc.hi, p);
  acc = df_quick(s.hi, __fadd_rn(s.lo, __fadd_rn(acc.lo, e)));
}

__device__ __forceinline__ dflt df_mul(dflt a, dflt b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_quick(p, e);
}

__device__ __forceinline__ dflt df_add(dflt a, dflt b) {
  const dflt s = df_two_sum(a.hi, b.hi);
  return df_quick(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ dflt df_split(double v) {
  const float h = __double2float_rn(v);
  return {h, __double2float_rn(v - (double)h)};
}

__device__ __forceinline__ double df_to_double(dflt v) { return (double)v.hi + (double)v.lo; }

__device__ __forceinline__ dflt df_neg(dflt a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ dflt df_sub(dflt a, dflt b) { return df_add(a, df_neg(b)); }
// a * b + c
__device__ __forceinline__ dflt df_madd(dflt a, dflt b, dflt c) {
  dflt acc = c;
  df_fma(acc, a.hi, a.lo, b.hi, b.lo);
  return acc;
}

// ---- double-float elementary functions (float units only)

// 1/sqrt(a), a > 0: float estimate, then two Newton steps y += y (1 - a y^2) / 2
// in double-float (each step doubles the correct bits, up to the format's ~48).
__device__ __forceinline__ dflt df_rsqrt(dflt a) {
  dflt y = {rsqrtf(a.hi), 0.f};
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const dflt e = df_sub({1.f, 0.f}, df_mul(a, df_mul(y, y)));
    y = df_madd(df_mul(y, {0.5f, 0.f}), e, y);
  }
  return y;
}

// Table of the double-float elementary functions (kDfmTableSize float2, hi/lo):
// [0, kErfcxIntervals * kErfcxTerms): Taylor coefficients of erfcx(x) =
// exp(x^2) erfc(x) at the centres of the intervals [i h, (i+1) h), h = 1/8;
// then exp(j/32) for j = -11 .. 11.
constexpr int kErfcxIntervals = 64, kErfcxTerms = 12;
constexpr float kErfcxMax = 8.f;  // x range covered: [0, 8]
constexpr int kExpTable = kErfcxIntervals * kErfcxTerms;
constexpr int kDfmTableSize = kExpTable + 23;

// exp(-y), y >= 0, by table-driven reduction (Tang, ACM TOMS 15, 1989):
// k = round(y / ln 2), t = k ln 2 - y (ln 2 split three ways, Cody & Waite, so
// k C1 is exact), j = round(32 t), s = t - j/32 (|s| <= 1/64);
// exp(-y) = 2^-k exp(j/32) exp(s), exp(s) by its Taylor series to s^7
// (remainder < 1e-19). Results below 2^-126 (y >= 87) are returned as 0.
__device__ __forceinline__ dflt df_exp_neg(dflt y, const float2* __restrict__ tab) {
  if (!(y.hi < 87.f)) return {0.f, 0.f};
  constexpr float kC1 = 6.931457520e-01f, kC2 = 1.428606765e-06f, kC3 = 5.495603972e-14f;
  const float k = rintf(y.hi * 1.44269502f);
  dflt t = df_add({k * kC1, 0.f}, df_neg(y));
  t = df_add(t, df_mul({k, 0.f}, {kC2, 0.f}));
  t = df_add(t, {k * kC3, 0.f});
  const float jf = rintf(t.hi * 32.f);
  const dflt s = df_add(t, {-jf * 0.03125f, 0.f});
  dflt p = {1.984127011e-04f, -2.725596875e-12f};                // 1/7!
  p = df_madd(p, s, {1.388888923e-03f, -3.363109444e-11f});      // 1/6!
  p = df_madd(p, s, {8.333333768e-03f, -4.346172033e-10f});      // 1/5!
  p = df_madd(p, s, {4.166666791e-02f, -1.241763470e-09f});      // 1/4!
  p = df_madd(p, s, {1.666666716e-01f, -4.967053879e-09f});      // 1/3!
  p = df_madd(p, s, {0.5f, 0.f});
  p = df_madd(p, s, {1.f, 0.f});
  p = df_madd(p, s, {1.f, 0.f});
  const float2 e = tab[kExpTable + 11 + (int)jf];
  const dflt r = df_mul(p, {e.x, e.y});
  const float sc = __int_as_float((127 - (int)k) << 23);  // 2^-k, k <= 126
  return {r.hi * sc, r.lo * sc};
}

// erfcx(x) = exp(x^2) erfc(x), 0 <= x <= 8: Taylor polynomial of the interval
// holding x (coefficients from the ODE y' = 2 x y - 2/sqrt(pi); see the host
// table builder), evaluated by Horner in double-float at t = x - centre.
__device__ __forceinline__ dflt df_erfcx(dflt x, const float2* __restrict__ tab) {
  const int i = max(0, min(kErfcxIntervals - 1, (int)(x.hi * 8.f)));
  const dflt t = df_add(x, {-((float)i + 0.5f) * 0.125f, 0.f});
  const float2* c = tab + i * kErfcxTerms;
  dflt p = {c[kErfcxTerms - 1].x, c[kErfcxTerms - 1].y};
#pragma unroll
  for (int n = kErfcxTerms - 2; n >= 0; --n) p = df_madd(p, t, {c[n].x, c[n].y});
  return p;
}

// Field at r of a multipole with kernels b1..b3, all double-float.
__device__ __forceinline__ void mp_field_df(const dflt r[3], const dflt* mp, dflt b1, dflt b2, dflt b3, dflt out[3]) {
  // mp: q, dx, dy, dz, Qxx, Qyy, Qzz, Qxy, Qxz, Qyz
  const dflt t0 = df_madd(mp[8], r[2], df_madd(mp[7], r[1], df_mul(mp[4], r[0])));
  const dflt t1 = df_madd(mp[9], r[2], df_madd(mp[5], r[1], df_mul(mp[7], r[0])));
  const dflt t2 = df_madd(mp[6], r[2], df_madd(mp[9], r[1], df_mul(mp[8], r[0])));
  const dflt rtr = df_madd(r[2], t2, df_madd(r[1], t1, df_mul(r[0], t0)));
  const dflt dr = df_madd(mp[3], r[2], df_madd(mp[2], r[1], df_mul(mp[1], r[0])));
  const dflt third = {0.333333343267f, -9.93410748e-09f};  // 1/3 = hi + lo
  const dflt two3 = {0.666666686535f, -1.98682150e-08f};   // 2/3 = hi + lo
  const dflt rad = df_madd(df_mul(b3, rtr), third, df_madd(b2, dr, df_mul(mp[0], b1)));
  const dflt c2 = df_mul(b2, two3);
  const dflt t[3] = {t0, t1, t2};
  for (int a = 0; a < 3; ++a) out[a] = df_sub(df_sub(df_mul(rad, r[a]), df_mul(b1, mp[1 + a])), df_mul(c2, t[a]));
}

// Sum over the kRowGroup lanes of one row; the mask names exactly this group.
__device__ __forceinline__ dflt df_group_sum(dflt v) {
  const unsigned mask = ((1u << kRowGroup) - 1u) << ((threadIdx.x & 31) & ~(kRowGroup - 1));
#pragma unroll
  for (int o = kRowGroup / 2; o > 0; o >>= 1) {
    dflt w;
    w.hi = __shfl_xor_sync(mask, v.hi, o, kRowGroup);
    w.lo = __shfl_xor_sync(mask, v.lo, o, kRowGroup);
    v = df_add(v, w);
  }
  return v;
}

}  // namespace amp

// ---- programmatic dependent launch (sm_90+): a kernel launched with
// launch_pdl may start while the previous kernel of its stream finishes; it
// calls pdl_wait() before touching anything that kernel writes (the wait
// returns once the previous grid has completed and its writes are visible),
// and pdl_trigger() to let its own successor be launched early. Kernels
// launched the ordinary way pass through pdl_wait() at once.
// 32-byte vector loads (sm_100 and later); p must be 32-byte aligned. The
// streaming form marks the lines evict-first; the read-only form goes
// through the non-coherent path (data the kernel does not write).
__device__ __forceinline__ void ld8_stream(const float4* p, float4& a, float4& b) {
  asm("ld.global.cs.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
      : "l"(p));
}
__device__ __forceinline__ void ld8_ro(const float4* p, float4& a, float4& b) {
  asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
      : "l"(p));
}

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" :::); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// launch geometry helpers
static inline int amp_blocks(long long work, int threads) {
  long long b = (work + threads - 1) / threads;
  return b < 1 ? 1 : (int)b;
}
