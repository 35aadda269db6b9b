// C ABI of libamoebapol (declared in include/amoebapol.h): context lifetime,
// system upload, and the calls that follow the paper's statement of the
// polarization problem (Section "Hotspots"): right-hand side (efld0_direct2),
// operator (tmatxb_pme2), solve, energy (epolar1).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "amp_internal.cuh"

namespace amp {

int dev_alloc_bytes(amp_ctx* c, void** p, size_t bytes) {
  *p = nullptr;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(c, AMP_ERR_OOM, "cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
  }
  c->allocs.push_back(*p);
  c->alloc_sizes.push_back(bytes);
  c->bytes += (long long)bytes;
  return AMP_OK;
}

void dev_free(amp_ctx* c, void* p) {
  if (!p) return;
  for (size_t k = 0; k < c->allocs.size(); ++k)
    if (c->allocs[k] == p) {
      c->allocs[k] = nullptr;
      c->bytes -= (long long)c->alloc_sizes[k];
      c->alloc_sizes[k] = 0;
    }
  cudaFree(p);
}

// Work of the context goes to stream st from now on (the serving layer moves
// pooled contexts between its workers' streams).
void ctx_bind_stream(amp_ctx* c, cudaStream_t st) {
  join_geometry(c);
  c->stream = st;
  if (c->plans) {
    cufftSetStream(c->plan_d2z, st);
    cufftSetStream(c->plan_z2d, st);
    if (c->plan_r2c) cufftSetStream(c->plan_r2c, st);
    if (c->plan_c2r) cufftSetStream(c->plan_c2r, st);
  }
}

constexpr int kEvPool = 8192;

// Each scope takes an event pair at begin and records its end into the same
// pair, so scopes may nest; events go on the stream the scope's launches use.
int prof_begin(amp_ctx* c, int phase, cudaStream_t st) {
  if (!c->prof) return -1;
  if (c->ev_used + 2 > (int)c->ev_pool.size()) {
    if (c->ev_open > 0) return -1;  // pool full inside an open scope: skip this one
    prof_resolve(c);
  }
  const int k = c->ev_used;
  c->ev_used += 2;
  c->ev_open += 1;
  cudaEventRecord(c->ev_pool[k], st);
  c->ev_phase[k / 2] = phase;
  return k;
}

void prof_end(amp_ctx* c, int slot, cudaStream_t st) {
  if (!c->prof || slot < 0) return;
  cudaEventRecord(c->ev_pool[slot + 1], st);
  c->ev_open -= 1;
}

int prof_resolve(amp_ctx* c) {
  if (c->ev_used == 0) return AMP_OK;
  int r = cuda_check(c, cudaStreamSynchronize(c->stream), "profile sync");
  if (r) return r;
  for (int k = 0; k < c->ev_used; k += 2) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev_pool[k], c->ev_pool[k + 1]);
    const int ph = c->ev_phase[k / 2];
    c->prof_ms[ph] += ms;
    c->prof_cnt[ph] += 1;
  }
  c->ev_used = 0;
  return AMP_OK;
}

int apply_T_sorted(amp_ctx* c, const double4_32a* v, const float4* v32, const float4* vlo, double4_32a* t,
                   double4_32a* t2);
void launch_to32(amp_ctx* c, const double4_32a* v, float4* o);

static int alloc_atoms(amp_ctx* c, int n) {
  if (n <= c->n_cap) return AMP_OK;
  void** bufs[] = {(void**)&c->cell_of, (void**)&c->perm, (void**)&c->inv_perm, (void**)&c->slot_tmp,
                   (void**)&c->atomA, (void**)&c->atomB, (void**)&c->atomC, (void**)&c->atomD,
                   (void**)&c->alph, (void**)&c->pos32, (void**)&c->full_cnt, (void**)&c->half_cnt,
                   (void**)&c->full_start, (void**)&c->half_start, (void**)&c->theta, (void**)&c->theta32,
                   (void**)&c->gbase, (void**)&c->E0s, (void**)&c->mu, (void**)&c->res, (void**)&c->zv,
                   (void**)&c->pv, (void**)&c->qv, (void**)&c->tv, (void**)&c->tmp, (void**)&c->p32,
                   (void**)&c->trec, (void**)&c->plo, (void**)&c->vhl, (void**)&c->mp_df, (void**)&c->wv,
                   (void**)&c->theta_df, (void**)&c->pd, (void**)&c->e0rec, (void**)&c->e0intra,
                   (void**)&c->xhl};
  for (void** b : bufs) {
    dev_free(c, *b);
    *b = nullptr;
  }
  const int cap = n;
  int r;
  if ((r = dev_alloc(c, &c->cell_of, cap)) || (r = dev_alloc(c, &c->perm, cap)) ||
      (r = dev_alloc(c, &c->inv_perm, cap)) || (r = dev_alloc(c, &c->slot_tmp, cap)) ||
      (r = dev_alloc(c, &c->atomA, cap)) || (r = dev_alloc(c, &c->atomB, cap)) ||
      (r = dev_alloc(c, &c->atomC, cap)) || (r = dev_alloc(c, &c->atomD, cap)) ||
      (r = dev_alloc(c, &c->alph, cap)) || (r = dev_alloc(c, &c->pos32, cap)) ||
      (r = dev_alloc(c, &c->full_cnt, cap)) || (r = dev_alloc(c, &c->half_cnt, cap)) ||
      (r = dev_alloc(c, &c->full_start, cap + 1)) || (r = dev_alloc(c, &c->half_start, cap + 1)) ||
      (r = pme_alloc_atoms(c, cap)) || (r = dev_alloc(c, &c->E0s, cap)) || (r = dev_alloc(c, &c->mu, cap)) ||
      (r = dev_alloc(c, &c->res, cap)) || (r = dev_alloc(c, &c->zv, cap)) || (r = dev_alloc(c, &c->pv, cap)) ||
      (r = dev_alloc(c, &c->qv, cap)) || (r = dev_alloc(c, &c->tv, cap)) || (r = dev_alloc(c, &c->tmp, cap)) ||
      (r = dev_alloc(c, &c->p32, cap)) || (r = dev_alloc(c, &c->trec, cap)) || (r = dev_alloc(c, &c->plo, cap)) ||
      (r = dev_alloc(c, &c->wv, cap)) || (r = dev_alloc(c, &c->vhl, 2LL * cap)) ||
      (r = dev_alloc(c, &c->mp_df, 5LL * cap)) || (r = dev_alloc(c, &c->pd, 3LL * cap)) ||
      (r = dev_alloc(c, &c->e0rec, cap)) || (r = dev_alloc(c, &c->e0intra, cap)) ||
      (r = dev_alloc(c, &c->xhl, 2LL * cap)))
    return r;
  c->n_cap = cap;
  return AMP_OK;
}

// The context stream waits for the geometry work that pme_geometry put on
// the side stream (once per new geometry).
void join_geometry(amp_ctx* c) {
  if (!c->geom_pending) return;
  cudaStreamWaitEvent(c->stream, c->ev_geom, 0);
  c->geom_pending = false;
}

}  // namespace amp

using namespace amp;

extern "C" {

int amp_create(amp_ctx** out, const amp_config* cfg, void* cuda_stream) {
  if (!out) return AMP_ERR_ARG;
  *out = nullptr;
  if (!cfg) return AMP_ERR_ARG;
  const bool cluster = cfg->box == 0.0;
  if (!(cfg->tol_debye > 0.0) || cfg->max_iter < 1 || (cfg->precision != AMP_FP64 && cfg->precision != AMP_MIXED))
    return AMP_ERR_ARG;
  if (!cluster && (!(cfg->box > 0.0) || !(cfg->cutoff > 0.0) || !(2.0 * cfg->cutoff < cfg->box) ||
                   !(cfg->ewald_beta > 0.0) || cfg->pme_grid < 8 || cfg->pme_grid > 512 || cfg->pme_order != kOrder ||
                   !(cfg->ewald_beta * cfg->cutoff <= (double)kErfcxMax)))
    return AMP_ERR_ARG;
  amp_ctx* c = new (std::nothrow) amp_ctx();
  if (!c) return AMP_ERR_OOM;
  c->cfg = *cfg;
  c->cluster = cluster;
  c->stream = (cudaStream_t)cuda_stream;
  int r;
  if ((r = dev_alloc(c, &c->flags, 4)) || (r = dev_alloc(c, &c->iflags, 8)) || (r = dev_alloc(c, &c->scal, 8)) ||
      (r = dev_alloc(c, &c->partials, 4 * kReduceBlocks)) || (r = dev_alloc(c, &c->vmax_part, kReduceBlocks + 2))) {
    amp_destroy(c);
    return r;
  }
  if (cudaMemset(c->vmax_part, 0, sizeof(float) * (kReduceBlocks + 2)) != cudaSuccess) {
    amp_destroy(c);
    return AMP_ERR_CUDA;
  }
  if (cudaHostAlloc((void**)&c->hbuf, 8 * sizeof(double), cudaHostAllocMapped) != cudaSuccess ||
      cudaHostAlloc((void**)&c->hibuf, 8 * sizeof(int), cudaHostAllocMapped) != cudaSuccess) {
    amp_destroy(c);
    return AMP_ERR_OOM;
  }
  if (cudaHostGetDevicePointer((void**)&c->hbuf_d, c->hbuf, 0) != cudaSuccess ||
      cudaHostGetDevicePointer((void**)&c->hibuf_d, c->hibuf, 0) != cudaSuccess) {
    amp_destroy(c);
    return AMP_ERR_CUDA;
  }
  // The reciprocal-space chain runs on the side stream beside the real-space
  // kernel and is the longer of the two: give its blocks priority.
  int prio_lo = 0, prio_hi = 0, dev = 0;
  cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || c->n_sm < 1)
    c->n_sm = 1;
  if (cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, prio_hi) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_geom, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_spread, cudaEventDisableTiming) != cudaSuccess) {
    amp_destroy(c);
    return AMP_ERR_CUDA;
  }
  if ((!cluster && (r = pme_setup(c))) || (r = dfm_setup(c))) {
    amp_destroy(c);
    return r;
  }
  *out = c;
  return AMP_OK;
}

int amp_reconfigure(amp_ctx* c, const amp_config* cfg) {
  if (!c || !cfg) return AMP_ERR_ARG;
  join_geometry(c);
  const bool cluster = cfg->box == 0.0;
  if (cluster != c->cluster || cfg->precision != c->cfg.precision)
    return fail(c, AMP_ERR_ARG, "amp_reconfigure: precision and cluster/periodic mode are fixed at creation");
  if (!(cfg->tol_debye > 0.0) || cfg->max_iter < 1) return fail(c, AMP_ERR_ARG, "amp_reconfigure: bad tolerance");
  if (!cluster && (cfg->pme_grid != c->cfg.pme_grid || cfg->pme_order != kOrder || !(cfg->box > 0.0) ||
                   !(cfg->cutoff > 0.0) || !(2.0 * cfg->cutoff < cfg->box) || !(cfg->ewald_beta > 0.0) ||
                   !(cfg->ewald_beta * cfg->cutoff <= (double)kErfcxMax)))
    return fail(c, AMP_ERR_ARG, "amp_reconfigure: same PME grid required, cutoff < box/2, 0 < beta cutoff <= 8");
  const bool box_changed = cfg->box != c->cfg.box || cfg->ewald_beta != c->cfg.ewald_beta;
  c->cfg = *cfg;
  c->have_system = false;
  c->skin_built = 0.0;
  if (2.0 * (c->cfg.cutoff + c->skin) >= c->cfg.box) c->skin = 0.0;
  if (!cluster && box_changed) return pme_influence(c);
  return AMP_OK;
}

void amp_destroy(amp_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  if (c->side) {
    cudaStreamSynchronize(c->side);
    cudaStreamDestroy(c->side);
  }
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->ev_geom) cudaEventDestroy(c->ev_geom);
  if (c->ev_spread) cudaEventDestroy(c->ev_spread);
  if (c->plan_d2z) cufftDestroy(c->plan_d2z);
  if (c->plan_z2d) cufftDestroy(c->plan_z2d);
  if (c->plan_r2c) cufftDestroy(c->plan_r2c);
  if (c->plan_c2r) cufftDestroy(c->plan_c2r);
  for (void* p : c->allocs)
    if (p) cudaFree(p);
  if (c->hbuf) cudaFreeHost(c->hbuf);
  if (c->hibuf) cudaFreeHost(c->hibuf);
  delete c;
}

const char* amp_last_error(const amp_ctx* c) { return c ? c->err : "null context"; }

int amp_set_system(amp_ctx* c, int n, const double* xyz, const double* q, const double* dip, const double* quad,
                   const double* alpha, const double* thole, const int* mol) {
  if (!c) return AMP_ERR_ARG;
  join_geometry(c);
  c->have_system = false;
  c->hist_len = c->hist_head = 0;  // a new system: no solution history
  if (n < 2 || !xyz || !q || !dip || !quad || !alpha || !thole || !mol)
    return fail(c, AMP_ERR_ARG, "amp_set_system: n >= 2 and all arrays are required");
  int r;
  if ((r = alloc_atoms(c, n))) return r;
  c->n = n;
  if (c->cluster) {
    if ((r = cluster_setup(c, xyz, q, dip, quad, alpha, thole, mol))) return r;
    c->have_system = true;
    return AMP_OK;
  }
  {
    PhaseScope ps(c, AMP_PHASE_LIST);
    if ((r = build_cells_and_lists(c, xyz, q, dip, quad, alpha, thole, mol))) return r;
  }
  {
    PhaseScope ps(c, AMP_PHASE_PAIR);
    launch_pair_build(c);
  }
  if ((r = cuda_check(c, cudaGetLastError(), "set_system launch"))) return r;
  c->have_system = true;
  return AMP_OK;
}

int amp_set_list_skin(amp_ctx* c, double skin) {
  if (!c) return AMP_ERR_ARG;
  if (c->cluster) return fail(c, AMP_ERR_ARG, "amp_set_list_skin: periodic contexts only");
  if (!(skin >= 0.0) || !(2.0 * (c->cfg.cutoff + skin) < c->cfg.box))
    return fail(c, AMP_ERR_ARG, "amp_set_list_skin: skin >= 0 with cutoff + skin < box/2");
  c->skin = skin;
  return AMP_OK;
}

int amp_update_positions(amp_ctx* c, const double* xyz, int* reused) {
  if (!c) return AMP_ERR_ARG;
  if (reused) *reused = 0;
  if (!c->have_system) return fail(c, AMP_ERR_STATE, "no system set");
  if (!xyz) return fail(c, AMP_ERR_ARG, "xyz is null");
  if (c->cluster) return fail(c, AMP_ERR_ARG, "amp_update_positions: periodic contexts only");
  join_geometry(c);
  bool ok = false;
  int r;
  {
    PhaseScope ps(c, AMP_PHASE_LIST);
    if ((r = reuse_lists(c, xyz, &ok))) return r;
  }
  if (!ok) return fail(c, AMP_ERR_STALE, "an atom moved more than skin/2 since amp_set_system (or no skin)");
  if ((r = pme_geometry(c))) return r;
  {
    PhaseScope ps(c, AMP_PHASE_PAIR);
    launch_pair_build(c);
  }
  if ((r = cuda_check(c, cudaGetLastError(), "update_positions launch"))) return r;
  if (reused) *reused = 1;
  return AMP_OK;
}

int amp_set_predictor(amp_ctx* c, int order) {
  if (!c) return AMP_ERR_ARG;
  if (order < -1 || order > 6) return fail(c, AMP_ERR_ARG, "amp_set_predictor: order in -1 .. 6");
  c->pred_order = order;
  c->hist_len = c->hist_head = 0;
  return AMP_OK;
}

int amp_permanent_field(amp_ctx* c, double* E0) {
  if (!c) return AMP_ERR_ARG;
  if (!c->have_system) return fail(c, AMP_ERR_STATE, "no system set");
  if (!E0) return fail(c, AMP_ERR_ARG, "E0 is null");
  if (c->cluster) {
    {
      PhaseScope ps(c, AMP_PHASE_E0_REAL);
      cluster_permanent_field(c, c->E0s);
    }
    launch_from_sorted(c, c->E0s, E0);
  } else {
    {
      PhaseScope ps(c, AMP_PHASE_E0_REAL);
      launch_e0_real(c, c->E0s);
    }
    join_geometry(c);  // the reciprocal part, computed beside the pair build
    launch_add_from_sorted(c, c->E0s, c->e0rec, E0);
  }
  return cuda_check(c, cudaGetLastError(), "permanent_field launch");
}

int amp_permanent_field_scaled(amp_ctx* c, double s_intra, double* E) {
  if (!c) return AMP_ERR_ARG;
  join_geometry(c);
  if (!c->have_system) return fail(c, AMP_ERR_STATE, "no system set");
  if (!E) return fail(c, AMP_ERR_ARG, "E is null");
  if (c->cluster) return fail(c, AMP_ERR_ARG, "amp_permanent_field_scaled: periodic contexts only");
  if (!(s_intra >= 0.0 && s_intra <= 1.0)) return fail(c, AMP_ERR_ARG, "amp_permanent_field_scaled: 0 <= s <= 1");
  {
    PhaseScope ps(c, AMP_PHASE_E0_REAL);
    launch_e0_real(c, c->E0s);
    if (s_intra != 0.0) launch_intra_scaled(c, s_intra, c->E0s);
  }
  join_geometry(c);
  launch_add_from_sorted(c, c->E0s, c->e0rec, E);
  return cuda_check(c, cudaGetLastError(), "permanent_field_scaled launch");
}

int amp_two_rhs_forces(amp_ctx* c, double s_intra, const double* mu_d, const double* mu_p, double* F, double* gq,
                       double* gdip, double* gquad) {
  if (!c) return AMP_ERR_ARG;
  join_geometry(c);
  if (!c->have_system) return fail(c, AMP_ERR_STATE, "no system set");
  if (!mu_d || !mu_p || !F) return fail(c, AMP_ERR_ARG, "mu_d, mu_p and F are required");
  if (c->cluster) return fail(c, AMP_ERR_ARG, "amp_two_rhs_forces: periodic contexts only");
  if (!(s_intra >= 0.0 && s_intra <= 1.0)) return fail(c, AMP_ERR_ARG, "amp_two_rhs_forces: 0 <= s <= 1");
  int r;
  if (c->tcg_cap < 4LL * c->n) {
    dev_free(c, c->tcg);
    c->tcg = nullptr;
    c->tcg_cap = 0;
    if ((r = dev_alloc(c, &c->tcg, 10LL * c->n))) return r;
    c->tcg_cap = 10LL * c->n;
  }
  double4_32a *md = c->tcg, *mp = md + c->n;
  launch_to_sorted(c, mu_d, md);
  launch_to_sorted(c, mu_p, mp);
  if ((r = two_rhs_forces(c, s_intra, md, mp, mp + c->n, F, gq, gdip, gquad))) return r;
  return cuda_check(c, cudaGetLastError(), "two_rhs_forces launch");
}

int amp_apply_T(amp_ctx* c, const double* mu, double* Tmu) {
  if (!c) return AMP_ERR_ARG;
  join_geometry(c);
  if (!c->have_system) return fail(c, AMP_ERR_STATE, "no system set");
  if (!mu || !Tmu) return fail(c, AMP_ERR_ARG, "null vector");
  launch_to_sorted(c, mu, c->tmp);
  float4* lo = c->cfg.precision == AMP_MIXED ? nullptr : c->plo;
  launch_split(c, c->tmp, c->p32, lo);
  int r = apply_T_sorted(c, c->tmp, c->p32, lo, c->tv, nullptr);
  if (r) return r;
  launch_from_sorted(c, c->tv, Tmu);
  return cuda_check(c, cudaGetLastError(), "apply_T launch");
}

int amp_solve_induced(amp_ctx* c, const double* E0, double* mu, int use_guess, int* iters, double* rms) {
  if (!c) return AMP_ERR_ARG;
  join_geometry(c);
  if (!c->have_system) return fail(c, AMP_ERR_STATE, "no system set");
  if (!E0 || !mu) return fail(c, AMP_ERR_ARG, "null vector");
  if (use_guess < 0 || use_guess > 2) return fail(c, AMP_ERR_ARG, "use_guess must be 0, 1 or 2");
  launch_to_sorted(c, E0, c->E0s);
  bool guess = use_guess == 1;
  if (use_guess == 1) launch_to_sorted(c, mu, c->mu);
  if (use_guess == 2) guess = predict_guess(c);
  int r = solve(c, guess);
  if (r != AMP_OK && r != AMP_ERR_NOT_CONVERGED) return r;
  if (r == AMP_OK) {
    const int e = push_history(c);
    if (e) return e;
  }
  launch_from_sorted(c, c->mu, mu);
  if (iters) *iters = c->stats.iters;
  if (rms) *rms = c->stats.rms;
  int e = cuda_check(c, cudaGetLastError(), "solve launch");
  return e ? e : r;
}

int amp_forces(amp_ctx* c, const double* mu, double* F, double* gq, double* gdip, double* gquad) {
  if (!c) return AMP_ERR_ARG;
  join_geometry(c);
  if (!c->have_system) return fail(c, AMP_ERR_STATE, "no system set");
  if (!mu || !F) return fail(c, AMP_ERR_ARG, "mu and F are required");
  if (c->cluster) return fail(c, AMP_ERR_ARG, "amp_forces: not available for isolated clusters");
  launch_to_sorted(c, mu, c->tmp);
  return forces(c, c->tmp, F, gq, gdip, gquad);
}

int amp_multipole_energy(amp_ctx* c, double* U, double* F, double* gq, double* gdip, double* gquad) {
  if (!c) return AMP_ERR_ARG;
  join_geometry(c);
  if (!c->have_system) return fail(c, AMP_ERR_STATE, "no system set");
  if (!U && !F && !gq && !gdip && !gquad) return fail(c, AMP_ERR_ARG, "amp_multipole_energy: no output requested");
  return multipole_energy(c, U, F, gq, gdip, gquad);
}

int amp_polarization_energy(amp_ctx* c, const double* mu, const double* E0, double* U) {
  if (!c) return AMP_ERR_ARG;
  join_geometry(c);
  if (!c->have_system) return fail(c, AMP_ERR_STATE, "no system set");
  if (!mu || !E0 || !U) return fail(c, AMP_ERR_ARG, "null pointer");
  return energy(c, mu, E0, U);
}

int amp_profile(amp_ctx* c, int enable) {
  if (!c) return AMP_ERR_ARG;
  if (enable) {
    if (c->ev_pool.empty()) {
      c->ev_pool.resize(kEvPool);
      c->ev_phase.resize(kEvPool / 2);
      for (auto& e : c->ev_pool)
        if (cudaEventCreate(&e) != cudaSuccess) return fail(c, AMP_ERR_CUDA, "cudaEventCreate failed");
    }
    c->ev_used = 0;
    for (int k = 0; k < AMP_NPHASE; ++k) {
      c->prof_ms[k] = 0.0;
      c->prof_cnt[k] = 0;
    }
    c->prof = true;
  } else {
    int r = prof_resolve(c);
    c->prof = false;
    return r;
  }
  return AMP_OK;
}

int amp_profile_read(amp_ctx* c, double* ms, long long* count) {
  if (!c || !ms || !count) return AMP_ERR_ARG;
  int r = prof_resolve(c);
  if (r) return r;
  for (int k = 0; k < AMP_NPHASE; ++k) {
    ms[k] = c->prof_ms[k];
    count[k] = c->prof_cnt[k];
  }
  return AMP_OK;
}

int amp_last_solve_stats(const amp_ctx* c, int* iters, int* fp64_checks) {
  if (!c) return AMP_ERR_ARG;
  if (iters) *iters = c->stats.iters;
  if (fp64_checks) *fp64_checks = c->stats.fp64_checks;
  return AMP_OK;
}

int amp_launch_count(const amp_ctx* c, long long* n) {
  if (!c || !n) return AMP_ERR_ARG;
  *n = c->n_launch;
  return AMP_OK;
}

int amp_pair_count(const amp_ctx* c, long long* n_pairs) {
  if (!c || !n_pairs) return AMP_ERR_ARG;
  *n_pairs = c->have_system ? c->n_half : 0;
  return AMP_OK;
}

}  // extern "C"
