// kernels.cuh -- launchers of the heat3d CUDA kernels (definitions in
// mg_kernels.cu and sdc_kernels.cu).  Every launcher enqueues on `st`,
// operates on `B` consecutive items at field stride g.fs (pointers address
// item 0 of the launch), skips item b when active != nullptr and active[b] == 0,
// and returns cudaGetLastError() of the launch.
#pragma once
#include "common.cuh"

namespace h3d {

// Launch shape of the stencil kernels.
// kind: 0 automatic (tiled for N >= 32, else z-march), 1 z-march (one column
// per thread), 2 shared-memory tile 32 x 8 (128 threads, 2 rows each), 3 tile
// 32 x 16 (256 threads, 2 rows each), 4 tile 32 x 16 (128 threads, 4 rows
// each), 5 and 6 as 2 and 3 with 6 planes of prefetch instead of 3; FP32
// Jacobi and residual only (all three stencils): four x points per thread, tile 128 x TY: 7 (4
// warps x 2 rows), 8 (8 warps x 1 row), 9 (4 warps x 4 rows), 10 (8 warps x
// 2 rows), 11 and 12 as 7 and 8 with 6 planes of prefetch, 13 as 7 with 10,
// 14 (2 warps x 2 rows, 6 planes); other operators take kind 3 for these; zc:
// planes per block along z.
struct Shape {
  int kind = 0;
  int zc = 16;
};

// Process-wide count of kernel launches (every launcher calls it once per launch).
void count_launch();

// ---- spatial operator (Sec. 1, method of lines) ----
// out = alpha_b * L u with L = (S1 - 6u) (order 2), (16 S1 - S2 - 90u)
// (order 4) or (2 S1 + S2 - 24 u) with S1 faces and S2 edges (compact, order
// kCompact); alpha_b = nu_b / h^2, nu_b / (12 h^2) or nu_b / (6 h^2).  When
// add_src != nullptr also writes add_dst = W u + add_src (the next substep's
// right-hand side; W = I but for the compact stencil, whose W u is also
// written to wu_out when given, at the stride of u).
cudaError_t launch_lap(int order, const Grid& g, int B, const double* u, long long u_stride,
                       double* out, long long out_stride, const double* alpha,
                       const double* add_src, double* add_dst, long long add_stride,
                       const int* active, Shape sh, cudaStream_t st, double* wu_out = nullptr);

// ---- multigrid pieces (Sec. 1.2) ----
// r = b - A u (FP64); bp_out = wd (TR) r, the scaled right-hand side of the
// error equation and the first Jacobi iterate (the V-cycle's levels hold
// b' = wd b, see Coef); norm_bits[b] = max(norm_bits[b], bits of max|r|)
// (optional).
template <typename TR>
cudaError_t launch_resid64(int order, const Grid& g, int B, const double* u, long long u_stride,
                           const double* b, long long b_stride, const Coef<double>* coef,
                           TR* bp_out, const Coef<TR>* coef_r,
                           unsigned long long* norm_bits, const int* active, Shape sh,
                           cudaStream_t st);

// Reads and clears the FP32 tile's lost-copy flag (synchronises the stream).
cudaError_t loader_timeouts_take(cudaStream_t st, int* flag);

// Damped Jacobi with the scaled right-hand side r = b' = wd b:
// out = e + wd (b - A e) = al e + be S (+ be2 S2) + b'.  With u64 != nullptr
// the result is added to u64 (u64 += out) instead of being stored in out.

template <typename T>
cudaError_t launch_jacobi(int order, const Grid& g, int B, const T* e, const T* r, T* out,
                          double* u64, long long u64_stride, const Coef<T>* coef,
                          const int* active, Shape sh, cudaStream_t st);

// rr = t' = wd (b - A e) = r - om e + be S (+ be2 S2), r = b' = wd b
template <typename T>
cudaError_t launch_resid(int order, const Grid& g, int B, const T* e, const T* r, T* rr,
                         const Coef<T>* coef, const int* active, Shape sh, cudaStream_t st);

// Exact solve on a one-unknown grid from the scaled right-hand side:
// e = r / a11w (= b / a11).
template <typename T>
cudaError_t launch_solve_one(const Grid& g, int B, const T* r, T* e, const Coef<T>* coef,
                             const int* active, cudaStream_t st);

// Full weighting of the scaled residual into the coarse level's scaled
// right-hand side: bc (coarse grid gc) <- rs * FW(rr) (fine grid gf,
// N_f = 2 N_c + 1; rs from the coarse level's coefficients cc).
template <typename T>
cudaError_t launch_restrict(const Grid& gf, const Grid& gc, int B, const T* rr, T* bc,
                            const Coef<T>* cc, const int* active, cudaStream_t st);

// Trilinear prolongation: uf = src + P ec (src may be uf: uf += P ec; both at
// the item stride uf_stride).
template <typename T>
cudaError_t launch_prolong_add(const Grid& gc, const Grid& gf, int B, const T* ec,
                               long long ec_stride, const T* src, T* uf, long long uf_stride,
                               const int* active, cudaStream_t st);

// uf += tensor-product npts-point midpoint interpolation of ec (the FAS
// correction with heat3d_config.interp = npts = 4, 6 or 8): along each axis
// even fine points take the coarse value, odd ones the npts-point Lagrange
// midpoint rule (4: (-e(I-1) + 9 e(I) + 9 e(I+1) - e(I+2)) / 16) on the odd
// extension of the coarse line about its zero boundary values.  FP64, B
// fields.  With scratch t1, t2 (each at least Nf * Nf * Nc doubles per field,
// field stride t_stride) it runs as three one-axis passes, bitwise the same,
// else as one point-wise kernel.
cudaError_t launch_prolong_add_mid(int npts, const Grid& gc, const Grid& gf, int B,
                                   const double* ec, long long ec_stride, double* uf,
                                   long long uf_stride, cudaStream_t st, double* t1 = nullptr,
                                   double* t2 = nullptr, long long t_stride = 0);

// The whole V-cycle below (and including) a level with N <= 15, one block per
// item, every level in shared memory (coarse_fused.cu).  Ns: sizes from that
// level down to 1; cf[l]: coefficients of level l for item 0 of the launch;
// b, e: the top level's right-hand side and correction (pitched, grid gtop).
constexpr int kFusedMaxN = 15;
template <typename T>
cudaError_t launch_vcycle_small(int order, int nlev, const int* Ns, const Coef<T>* const* cf,
                                int B, const T* b, T* e, const Grid& gtop, int nu1, int nu2,
                                const int* active, cudaStream_t st);

// The whole solve of mg_vcycle's rule for B items on a grid with 15 <= N <=
// kPersistMaxN (orders 2 and 4) as one persistent cooperative kernel
// (persist.cu): FP64 residual and norm, `inner` V(nu1, nu2) cycles per
// residual, the stop rule of launch_mg_check after each residual, until every
// item has stopped or max_cycles cycles ran; bitwise the results of the
// launch sequence.  Pointers address item 0 of the launch; the multigrid
// fields of level k are at stride g[k].fs, u and rhs (FP64, grid g[0]) at
// strides us and bs.  active: B flags, 1 on entry; ncyc and nan_flag zeroed by
// the caller; tol, last as launch_mg_check; norm2: 2 B scratch words and ctl:
// 4 words of barrier state, both zeroed here.  ctl[1] is set when a grid
// barrier gave up waiting (about 1 s), and the kernel then returned early.
constexpr int kPersistMaxN = 63;
template <typename T>
struct MgPersist {
  int nlev;  // multigrid levels, g[nlev - 1].N == 1
  Grid g[kMaxLevels];
  T* b[kMaxLevels];
  T* e[kMaxLevels];
  T* t[kMaxLevels];
  const Coef<T>* cf[kMaxLevels];
  const Coef<double>* c64;
  double* u;
  long long us;
  const double* rhs;
  long long bs;
  int B, nu1, nu2, inner, max_cycles;
  unsigned long long* norm2;
  int* active;
  int* ncyc;
  double* last;
  const double* tol;
  int* nan_flag;
  int* ctl;
};
bool mg_persist_supported(int order, int N);
template <typename T>
cudaError_t launch_mg_persist(int order, const MgPersist<T>& p, cudaStream_t st);

// u64 += e
template <typename T>
cudaError_t launch_update(const Grid& g, int B, const T* e, double* u64, long long u64_stride,
                          const int* active, cudaStream_t st);

// Device-side stop rule of a multigrid solve after a residual: per item b that
// is active, last[b] = its residual norm (from norm_bits); init: deactivate
// items already at tol; else count the cycle (ncyc[b]++) and deactivate at
// norm <= tol[b] or ncyc[b] >= *max_cycles (device memory, so that a captured
// graph serves any cap).  A NaN/Inf norm deactivates the item and sets *nan_flag.
cudaError_t launch_mg_check(int B, const unsigned long long* norm_bits, int* active,
                            const double* tol, int* ncyc, double* last, const int* max_cycles,
                            int* nan_flag, bool init, cudaStream_t st);

// max|u| per item into norm_bits (bits of the double), FP64 input.
cudaError_t launch_maxabs(const Grid& g, int B, const double* u, long long u_stride,
                          unsigned long long* norm_bits, const int* active, cudaStream_t st);

// ---- layout and copies ----
cudaError_t launch_dense_to_pitched(const Grid& g, int B, const double* dense, double* f,
                                    long long f_stride, cudaStream_t st);
cudaError_t launch_pitched_to_dense(const Grid& g, int B, const double* f, long long f_stride,
                                    double* dense, cudaStream_t st);
// dst_b = src_b for B items (item strides may differ, e.g. node 0 of slice p
// from node M-1 of slice p-1).
cudaError_t launch_copy(const Grid& g, int B, const double* src, long long src_stride,
                        double* dst, long long dst_stride, cudaStream_t st);

// ---- SDC (Sec. 1.1) ----
// For item b with nodes U_0..U_{M-1}, F_0..F_{M-1} (node stride g.fs, item
// stride M g.fs):
//   J_m  = sum_j dtS[m][j] F_j + gS[m] Phi + tauS_m         (m = 0..M-2)
//   I_m  = J_m - dtm[m] F_{m+1}      written to I (item stride (M-1) g.fs)
//   I_0 += U_0                        (right-hand side of the first substep)
//   residual (optional): max over m of |U_0 + sum_{m' <= m} J_{m'} - U_{m+1}|
cudaError_t launch_integrals(int M, const Grid& g, int B, const double* U, const double* F,
                             const double* tauS, double* I, const ItemSDC* items,
                             const double* phi1d, unsigned long long* res_bits,
                             const int* active, cudaStream_t st);

// ---- FAS (Sec. 1.1) ----
// Injection of the fine nodes onto the coarse level and the fine Q-integral:
//   UG_m = UGr_m = R UF_{jm},  qF_m = R(sum_j dtQ^F[jm][j] F^F_j) + gQ^F[jm] Phi
// Compact fine level: X (field m-1 of each item at stride xs, for coarse node
// m >= 1) holds W^{-1} r, and qF_m = R(U_jm - U_0 + X_{m-1}) instead.
cudaError_t launch_fas_inject(int MF, int MG, const Grid& gf, const Grid& gg, int B,
                              const double* UF, const double* FF, double* UG, double* UGr,
                              double* qF, const ItemSDC* itF, const FasMap* map,
                              const double* phig1d, cudaStream_t st, const double* X = nullptr,
                              long long xs = 0);
// Compact fine level, fine node jm: weighted residual
// r = W U_0 + sum_p dtQ[jm][p] F_p + gQ[jm] Phi - W U_jm into R (one field per
// item) and X (item stride xs); max |r| per item into res_bits (zeroed by the caller).
cudaError_t launch_fas_wresid(int MF, const Grid& gf, int B, int jm, const double* WU,
                              const double* FF, const ItemSDC* itF, const double* phif1d,
                              double* R, double* X, long long xs, unsigned long long* res_bits,
                              cudaStream_t st);
// tauQ_m = qF_m - sum_i dtQ^G[m][i] F^G_i - gQ^G[m] Phi;  tauS_m = tauQ_{m+1} - tauQ_m
cudaError_t launch_fas_tau(int MG, const Grid& gg, int B, const double* qF, const double* FG,
                           double* tauS, const ItemSDC* itG, const double* phig1d,
                           cudaStream_t st);
// D_j = sum_m L[j][m] (UG_m - UGr_m) on the coarse grid (MF fields per item).
cudaError_t launch_fas_delta(int MF, int MG, const Grid& gg, int B, const double* UG,
                             const double* UGr, double* D, const FasMap* map, cudaStream_t st);

}  // namespace h3d
