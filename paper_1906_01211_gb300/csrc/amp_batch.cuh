// Records of the batched small-cluster engine (amp_batch.cu), shared with the
// server that drives it (amp_server.cu).
#pragma once

#include "amp_internal.cuh"

namespace amp {
namespace batch {

constexpr int kRows = 64;      // rows of one work item (a tile of a request's atoms)
constexpr int kThreads = 128;  // two threads per row
constexpr int kChunk = 128;    // columns staged in shared memory at a time

// what the pair phase does next for a request (ReqT.kind)
enum Kind { K_E0 = 0, K_INIT = 1, K_ITER = 2, K_AFTER = 3, K_DONE = 4 };
// what a phase does for a request in one launch (ReqS.act)
enum Act { A_IDLE = 0, A_E0 = 1, A_TV = 2, A_TVI = 3, A_CHECK = 4, A_FINISH = 5 };

struct ReqInfo {  // written by the host at admission
  int off, n, tile0, ntiles;  // arena atom offset (multiple of kRows), atoms, first tile, tiles
  double tol;
  int max_iter, pad;
};

struct ReqT {  // written by the vector phase (tile 0) and the host, read by the pair phase
  int kind, iter, first, pad;
  double rho, gamma;
};

struct ReqS {  // written by the pair phase (tile 0), read by the vector phase
  int act, iter, first, pad;
  double rho_old, gamma_old, rms;
};

struct ReqOut {  // written once the request has ended
  int status, iters;  // status 0 running, 1 converged, 2 iteration cap, 3 breakdown
  double rms, U;
};

// Device arrays of one engine (per atom of the arena, per request slot, per tile).
struct Arena {
  float4* p32;    // (x, y, z, 1/sqrt(alpha))
  float2* tm32;   // (thole, molecule as int bits)
  float4* mp32;   // 3 per atom: (q, dx, dy, dz), (Qxx, Qyy, Qzz, Qxy), (Qxz, Qyz, 0, 0)
  float4* pdf;    // 3 per atom: hi (x, y, z, 1/sqrt(alpha)), lo of the same, (thole hi, lo, molecule, 0)
  float4* v32;    // the float32 operator input
  double2* al;    // (alpha, 1/alpha)
  double4_32a *e0, *mu, *r, *z, *p, *q, *w, *tmp;
  double *part_rz, *part_zw, *partz, *parte;  // per tile
  ReqInfo* info;
  ReqT* reqT;
  ReqS* reqS;
  ReqOut* out;
};

__global__ void k_batch_pairs(Arena A, int n_items, const int2* __restrict__ items, int* __restrict__ heads,
                              const float2* __restrict__ tab);
__global__ void k_batch_vectors(Arena A, int n_items, const int2* __restrict__ items, int* __restrict__ heads);
__global__ void k_batch_records(int off, int n, const double* __restrict__ xyz, const double* __restrict__ q,
                                const double* __restrict__ dip, const double* __restrict__ quad,
                                const double* __restrict__ alpha, const double* __restrict__ thole,
                                const int* __restrict__ mol, Arena A, int* __restrict__ bad);
__global__ void k_batch_result(int off, int n, const double4_32a* __restrict__ mu, double* __restrict__ out);

}  // namespace batch
}  // namespace amp
