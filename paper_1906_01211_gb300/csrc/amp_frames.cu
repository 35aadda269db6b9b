// Local-frame multipoles and the forces from their frames.
//
// AMOEBA (the force field of the paper's Section "Polarizable AMOEBA force
// field") gives each site's dipole and quadrupole in a local frame fixed by
// two neighbouring atoms, so the global moments turn with the molecule
// (Ren & Ponder's conventions). For site i with axis atoms zi and xi,
// v1 = x_zi - x_i, v2 = x_xi - x_i:
//   Z-then-X (kind 0): e_z = v1/|v1|;  bisector (kind 1): e_z = a/|a|,
//   a = v1/|v1| + v2/|v2|; then b = v2 - (v2.e_z) e_z, e_x = b/|b|,
//   e_y = e_z x e_x; R = [e_x e_y e_z] (columns);
//   d = R d_loc, Theta = R Theta_loc R^T.
// With moments tied to frames, an energy's forces gain the frame terms
//   F_k -= sum_i [ dU/dd_i . dR d_loc + dU/dTheta_i : (dR Theta_loc R^T + R Theta_loc dR^T) ],
// dR/dx_k from d(v/|v|) = (I - e e^T) dv/|v| and the product rule (k = i,
// zi, xi). A site whose kind is not 0 or 1, or whose axis atoms are not two
// other atoms of the system, keeps its moments as given and adds no force.
// The moment gradients dU/dd, dU/dTheta are those of amp_forces,
// amp_multipole_energy or amp_tcg1 (at fixed frames). Context-free calls on
// a stream; caller order, device arrays; float64 throughout (few operations
// per site).
#include "amp_internal.cuh"

namespace amp {
namespace {

struct M3 {
  double m[3][3];
};

__device__ __forceinline__ void unit(const double v[3], double e[3], double& n) {
  n = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  for (int a = 0; a < 3; ++a) e[a] = v[a] / n;
}

__device__ __forceinline__ double dot3(const double a[3], const double b[3]) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

__device__ __forceinline__ void cross3(const double a[3], const double b[3], double c[3]) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

// The frame of site i and what its derivatives need.
struct Frame {
  double v1[3], v2[3], u1[3], u2[3], n1, n2, a[3], na, ez[3], b[3], nb, ex[3], ey[3];
  int kind;
};

__device__ __forceinline__ void frame_of(const double* xyz, int i, int zi, int xi, int kind, Frame& f) {
  f.kind = kind;
  for (int c = 0; c < 3; ++c) {
    f.v1[c] = xyz[3 * zi + c] - xyz[3 * i + c];
    f.v2[c] = xyz[3 * xi + c] - xyz[3 * i + c];
  }
  unit(f.v1, f.u1, f.n1);
  unit(f.v2, f.u2, f.n2);
  for (int c = 0; c < 3; ++c) f.a[c] = kind == 1 ? f.u1[c] + f.u2[c] : f.v1[c];
  unit(f.a, f.ez, f.na);
  const double p = dot3(f.v2, f.ez);
  for (int c = 0; c < 3; ++c) f.b[c] = f.v2[c] - p * f.ez[c];
  unit(f.b, f.ex, f.nb);
  cross3(f.ez, f.ex, f.ey);
}

__device__ __forceinline__ M3 rot(const Frame& f) {  // columns e_x, e_y, e_z
  M3 R;
  for (int r = 0; r < 3; ++r) {
    R.m[r][0] = f.ex[r];
    R.m[r][1] = f.ey[r];
    R.m[r][2] = f.ez[r];
  }
  return R;
}

// dR for a displacement of v1 by dv1 and of v2 by dv2
__device__ __forceinline__ M3 drot(const Frame& f, const double dv1[3], const double dv2[3]) {
  double da[3];
  if (f.kind == 1) {
    const double p1 = dot3(f.u1, dv1), p2 = dot3(f.u2, dv2);
    for (int c = 0; c < 3; ++c) da[c] = (dv1[c] - f.u1[c] * p1) / f.n1 + (dv2[c] - f.u2[c] * p2) / f.n2;
  } else {
    for (int c = 0; c < 3; ++c) da[c] = dv1[c];
  }
  double dez[3];
  const double pa = dot3(f.ez, da);
  for (int c = 0; c < 3; ++c) dez[c] = (da[c] - f.ez[c] * pa) / f.na;
  const double v2ez = dot3(f.v2, f.ez), dv2ez = dot3(dv2, f.ez), v2dez = dot3(f.v2, dez);
  double db[3];
  for (int c = 0; c < 3; ++c) db[c] = dv2[c] - dv2ez * f.ez[c] - v2dez * f.ez[c] - v2ez * dez[c];
  double dex[3];
  const double pb = dot3(f.ex, db);
  for (int c = 0; c < 3; ++c) dex[c] = (db[c] - f.ex[c] * pb) / f.nb;
  double t1[3], t2[3];
  cross3(dez, f.ex, t1);
  cross3(f.ez, dex, t2);
  M3 D;
  for (int r = 0; r < 3; ++r) {
    D.m[r][0] = dex[r];
    D.m[r][1] = t1[r] + t2[r];
    D.m[r][2] = dez[r];
  }
  return D;
}

__device__ __forceinline__ void quad_mat(const double* q6, double T[3][3]) {
  T[0][0] = q6[0];
  T[1][1] = q6[1];
  T[2][2] = q6[2];
  T[0][1] = T[1][0] = q6[3];
  T[0][2] = T[2][0] = q6[4];
  T[1][2] = T[2][1] = q6[5];
}

// A T B^T for 3x3 (A, B as M3)
__device__ __forceinline__ void sandwich(const M3& A, const double T[3][3], const M3& B, double out[3][3]) {
  double AT[3][3];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) AT[r][c] = A.m[r][0] * T[0][c] + A.m[r][1] * T[1][c] + A.m[r][2] * T[2][c];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) out[r][c] = AT[r][0] * B.m[c][0] + AT[r][1] * B.m[c][1] + AT[r][2] * B.m[c][2];
}

// A site has a frame when its kind is 0 or 1 and both axis atoms are other
// atoms of the system (any other site keeps its moments as given).
__device__ __forceinline__ bool framed(int i, int n, const int* kind, const int* zatom, const int* xatom) {
  const int k = kind[i], zi = zatom[i], xi = xatom[i];
  return (k == 0 || k == 1) && zi >= 0 && zi < n && xi >= 0 && xi < n && zi != i && xi != i && zi != xi;
}

__global__ void k_frames_global(int n, const double* __restrict__ xyz, const double* __restrict__ dloc,
                                const double* __restrict__ qloc, const int* __restrict__ kind,
                                const int* __restrict__ zatom, const int* __restrict__ xatom,
                                double* __restrict__ dip, double* __restrict__ quad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (!framed(i, n, kind, zatom, xatom)) {
    for (int c = 0; c < 3; ++c) dip[3 * i + c] = dloc[3 * i + c];
    for (int c = 0; c < 6; ++c) quad[6 * i + c] = qloc[6 * i + c];
    return;
  }
  Frame f;
  frame_of(xyz, i, zatom[i], xatom[i], kind[i], f);
  const M3 R = rot(f);
  for (int r = 0; r < 3; ++r)
    dip[3 * i + r] = R.m[r][0] * dloc[3 * i] + R.m[r][1] * dloc[3 * i + 1] + R.m[r][2] * dloc[3 * i + 2];
  double T[3][3], G[3][3];
  quad_mat(qloc + 6 * i, T);
  sandwich(R, T, R, G);
  quad[6 * i] = G[0][0];
  quad[6 * i + 1] = G[1][1];
  quad[6 * i + 2] = G[2][2];
  quad[6 * i + 3] = G[0][1];
  quad[6 * i + 4] = G[0][2];
  quad[6 * i + 5] = G[1][2];
}

// F_k -= sum over framed sites i of dU/dM_i . dM_i/dx_k (k = i, zi, xi), one
// thread per site, float64 atomics into F (each atom gets contributions from
// the sites whose frames it fixes).
__global__ void k_frame_forces(int n, const double* __restrict__ xyz, const double* __restrict__ dloc,
                               const double* __restrict__ qloc, const int* __restrict__ kind,
                               const int* __restrict__ zatom, const int* __restrict__ xatom,
                               const double* __restrict__ gd, const double* __restrict__ gt,
                               double* __restrict__ F) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || !framed(i, n, kind, zatom, xatom)) return;
  Frame f;
  const int zi = zatom[i], xi = xatom[i];
  frame_of(xyz, i, zi, xi, kind[i], f);
  const M3 R = rot(f);
  double T[3][3];
  quad_mat(qloc + 6 * i, T);
  const double dl[3] = {dloc[3 * i], dloc[3 * i + 1], dloc[3 * i + 2]};
  const double g_d[3] = {gd[3 * i], gd[3 * i + 1], gd[3 * i + 2]};
  const double* g6 = gt + 6 * i;
  const int atoms[3] = {i, zi, xi};
  const double s1[3] = {-1.0, 1.0, 0.0}, s2[3] = {-1.0, 0.0, 1.0};
  for (int k = 0; k < 3; ++k)
    for (int c = 0; c < 3; ++c) {
      double dv1[3] = {0.0, 0.0, 0.0}, dv2[3] = {0.0, 0.0, 0.0};
      dv1[c] = s1[k];
      dv2[c] = s2[k];
      const M3 D = drot(f, dv1, dv2);
      double dd = 0.0;
      for (int r = 0; r < 3; ++r) dd += g_d[r] * (D.m[r][0] * dl[0] + D.m[r][1] * dl[1] + D.m[r][2] * dl[2]);
      double A[3][3], B[3][3];
      sandwich(D, T, R, A);  // dR Theta R^T
      sandwich(R, T, D, B);  // R Theta dR^T
      const double dth[6] = {A[0][0] + B[0][0], A[1][1] + B[1][1], A[2][2] + B[2][2],
                             A[0][1] + B[0][1], A[0][2] + B[0][2], A[1][2] + B[1][2]};
      double dq = 0.0;
      for (int m = 0; m < 6; ++m) dq += g6[m] * dth[m];
      atomicAdd(F + 3 * atoms[k] + c, -(dd + dq));
    }
}

}  // namespace
}  // namespace amp

using namespace amp;

extern "C" int amp_frames_to_global(int n_atoms, const double* xyz, const double* dip_local,
                                    const double* quad_local, const int* kind, const int* zatom, const int* xatom,
                                    double* dip, double* quad, void* cuda_stream) {
  if (n_atoms < 1 || !xyz || !dip_local || !quad_local || !kind || !zatom || !xatom || !dip || !quad)
    return AMP_ERR_ARG;
  if (cudaPeekAtLastError() != cudaSuccess) return AMP_ERR_CUDA;
  k_frames_global<<<amp_blocks(n_atoms, 128), 128, 0, static_cast<cudaStream_t>(cuda_stream)>>>(
      n_atoms, xyz, dip_local, quad_local, kind, zatom, xatom, dip, quad);
  if (cudaPeekAtLastError() != cudaSuccess) {
    cudaGetLastError();
    return AMP_ERR_CUDA;
  }
  return AMP_OK;
}

extern "C" int amp_frame_forces(int n_atoms, const double* xyz, const double* dip_local, const double* quad_local,
                                const int* kind, const int* zatom, const int* xatom, const double* gdip,
                                const double* gquad, double* F, void* cuda_stream) {
  if (n_atoms < 1 || !xyz || !dip_local || !quad_local || !kind || !zatom || !xatom || !gdip || !gquad || !F)
    return AMP_ERR_ARG;
  if (cudaPeekAtLastError() != cudaSuccess) return AMP_ERR_CUDA;
  k_frame_forces<<<amp_blocks(n_atoms, 128), 128, 0, static_cast<cudaStream_t>(cuda_stream)>>>(
      n_atoms, xyz, dip_local, quad_local, kind, zatom, xatom, gdip, gquad, F);
  if (cudaPeekAtLastError() != cudaSuccess) {
    cudaGetLastError();
    return AMP_ERR_CUDA;
  }
  return AMP_OK;
}
