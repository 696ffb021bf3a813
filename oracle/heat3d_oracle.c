/*
 * heat3d_oracle.c -- plain, slow FP64 CPU oracle for the SDC / MLSDC / PFASST
 * solver of the forced 3-D heat equation (Speck, Ruprecht, Emmett, Bolten,
 * Krause, arXiv:1307.7867).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark load this library.  The product path
 * (libheat3d.so) shares no code, header, table or constant generator with it.
 *
 * Everything is FP64 with straightforward loops, in the order the paper states
 * the method.  The per-point loops carry OpenMP pragmas: the parity oracle is
 * built without OpenMP (one thread; the pragmas are ignored), and a second
 * build with -fopenmp only times the CPU baseline on all host cores.  Every
 * point is computed by the same expression in either build, so the two give
 * bitwise equal results (tested); reductions stay serial.  Grid functions are dense N^3 arrays of interior values,
 * x fastest, z slowest; interior indices i, j, k run 1..N, h = 1/(N+1),
 * x_i = i*h, and u = 0 on the boundary (Sec. 1, Eqs. 1-2).
 *
 * Readings of points the paper leaves open (all stated once more at the
 * function that uses them):
 *   - fine stencil: 4th-order "wide" 13-point Laplacian with odd-reflection
 *     ghosts u_{-1} = -u_1, u_{N+2} = -u_N (order 4), or the 4th-order compact
 *     19-point Mehrstellen operator (order 19, Sec. 1 and Sec. 1.2): the
 *     semi-discrete system is W u' = nu L u + W f with the weighting matrix
 *     W = I + (h^2/12) Delta_7; SDC runs in that weighted form and the FAS
 *     restriction maps the fine integrals back by W^{-1} (multigrid);
 *   - M counts Gauss-Lobatto nodes including both ends of the step;
 *   - multigrid: damped Jacobi (omega 6/7 for 7 points, 9/11 for 13 points,
 *     12/11 for the compact operator, constant interior diagonal),
 *     full-weighting restriction, trilinear
 *     prolongation, rediscretised coarse operators, N -> (N-1)/2 down to one
 *     unknown solved exactly (Sec. 1.2);
 *   - solve stop rule: max|b - A u| <= tol, checked before every cycle;
 *   - SDC initial iterate: the initial value spread to every node;
 *   - FAS: injection in space and time, trilinear (or, with interp = 4, 6,
 *     8, the tensor-product 4-, 6- or 8-point midpoint rule) + Lagrange
 *     interpolation in time of the coarse correction; PFASST schedule and
 *     predictor as coded below, pinned by its converged limit (the serial
 *     collocation solution), by the one-slice case equal to MLSDC, and at a
 *     fixed iteration count by a scalar recursion of the same schedule on one
 *     sine mode (both levels on one mesh, every node of every slice after 1-3
 *     iterations) and by causality (slice 0 equals MLSDC's first step; the
 *     first slices of a run equal a shorter run);
 *   - optional solver tolerance tied to the sweep's incoming residual
 *     (mg_rel), and the W-solve of the compact FAS restriction applied to the
 *     weighted residual (U_j - U_0 + W^{-1} r), see or_fas_restrict_st.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_EINVAL (-1)
#define OR_ENOMEM (-2)
#define OR_ENOTCONV (-3)

#define OR_PI 3.14159265358979323846
#define OR_COMPACT 19 /* order code of the compact 19-point stencil */
/* The W-solve of the FAS restriction stops at max(mg_tol, OR_W_REL * |r|). */
#define OR_W_REL 1e-2

typedef struct {
  int N;     /* interior points per axis */
  int order; /* 2: 7-point Laplacian, 4: 13-point wide Laplacian, 19: compact */
  int M;     /* Gauss-Lobatto nodes per step, both end points included */
} or_level;

typedef struct {
  double nu;      /* diffusion coefficient (nu = 0.1 in Sec. 1) */
  int forcing;    /* 0: f = 0; 1: f = -Phi(x) (sin t - kappa nu pi^2 cos t) */
  double kappa;   /* 1: forcing as printed in Eq. 3; 3: exact for Eq. 4 */
  double mg_tol;  /* stop a solve when max|b - A u| <= mg_tol; < 0: fixed count */
  int mg_max;     /* V-cycle cap per solve */
  int nu1, nu2;   /* pre- and post-smoothing sweeps, V(nu1, nu2) */
  double mg_rel;  /* > 0: a sweep's solves stop at max(mg_tol, mg_rel * residual of the
                     sweep's incoming iterate) */
  int interp;     /* spatial interpolation of the FAS correction: 4, 6, 8 = the
                     tensor-product 4-, 6- or 8-point midpoint rule (odd extension
                     about the boundary), else trilinear */
} or_problem;

typedef struct {
  long vcycles;    /* V-cycles over all solves */
  long solves;     /* implicit solves */
  long sweeps;     /* SDC sweeps on any level */
  long iters;      /* MLSDC / PFASST iterations */
  double residual; /* last SDC / PFASST residual computed */
  int notconv;     /* number of solves that hit the cycle cap */
  double vcycle_points; /* sum over V-cycles of the solved grid's N^3 (work count) */
} or_stats;

static size_t n3(int N) { return (size_t)N * N * N; }
static size_t id3(int N, int i, int j, int k) {
  return (((size_t)(k - 1) * N + (j - 1)) * N + (i - 1));
}

/* ------------------------------------------------------------------------ */
/* Spatial discretisation (Sec. 1: method of lines, 2nd- and 4th-order)      */
/* ------------------------------------------------------------------------ */

/* One axis index with the boundary rule: 0 and N+1 are Dirichlet zeros; the
 * wide stencil's ghosts -1 and N+2 mirror 1 and N with a sign change.
 * Returns 0 for a zero value, else the interior index and its sign. */
static int axis_index(int N, int a, int* sign) {
  if (a == 0 || a == N + 1) return 0;
  if (a == -1) { *sign = -*sign; return 1; }
  if (a == N + 2) { *sign = -*sign; return N; }
  return a;
}

static double value_at(const double* u, int N, int i, int j, int k) {
  int s = 1;
  int ii = axis_index(N, i, &s);
  int jj = axis_index(N, j, &s);
  int kk = axis_index(N, k, &s);
  if (ii == 0 || jj == 0 || kk == 0) return 0.0;
  return s * u[id3(N, ii, jj, kk)];
}

/* Compact (Mehrstellen) Laplacian L u = (1/(6 h^2)) (-24 u + 2 * (sum of the
 * 6 face neighbours) + (sum of the 12 edge neighbours)), zero boundary. */
static void compact_laplacian(int N, const double* u, double* out) {
  double h = 1.0 / (N + 1);
  #pragma omp parallel for
  for (int k = 1; k <= N; ++k)
    for (int j = 1; j <= N; ++j)
      for (int i = 1; i <= N; ++i) {
        double faces = 0.0, edges = 0.0;
        for (int dk = -1; dk <= 1; ++dk)
          for (int dj = -1; dj <= 1; ++dj)
            for (int di = -1; di <= 1; ++di) {
              int nz = (di != 0) + (dj != 0) + (dk != 0);
              double v = value_at(u, N, i + di, j + dj, k + dk);
              if (nz == 1) faces += v;
              if (nz == 2) edges += v;
            }
        out[id3(N, i, j, k)] = (-24.0 * u[id3(N, i, j, k)] + 2.0 * faces + edges) / (6.0 * h * h);
      }
}

/* out = W u: the weighting matrix of the compact scheme,
 * (6 u + sum of the 6 face neighbours) / 12 = u + (h^2 / 12) Delta_7 u; the
 * identity for the other stencils. */
void or_weight(int N, int order, const double* u, double* out) {
  if (order != OR_COMPACT) { memcpy(out, u, n3(N) * sizeof(double)); return; }
  #pragma omp parallel for
  for (int k = 1; k <= N; ++k)
    for (int j = 1; j <= N; ++j)
      for (int i = 1; i <= N; ++i) {
        double faces = value_at(u, N, i - 1, j, k) + value_at(u, N, i + 1, j, k) +
                       value_at(u, N, i, j - 1, k) + value_at(u, N, i, j + 1, k) +
                       value_at(u, N, i, j, k - 1) + value_at(u, N, i, j, k + 1);
        out[id3(N, i, j, k)] = (6.0 * u[id3(N, i, j, k)] + faces) / 12.0;
      }
}

/* out = Delta_h u.  order 2: (u_{-1} - 2 u + u_{+1}) / h^2 per axis;
 * order 4: (-u_{-2} + 16 u_{-1} - 30 u + 16 u_{+1} - u_{+2}) / (12 h^2);
 * order 19: the compact operator L (W^{-1} L approximates Delta). */
void or_laplacian(int N, int order, const double* u, double* out) {
  if (order == OR_COMPACT) { compact_laplacian(N, u, out); return; }
  double h = 1.0 / (N + 1);
  #pragma omp parallel for
  for (int k = 1; k <= N; ++k)
    for (int j = 1; j <= N; ++j)
      for (int i = 1; i <= N; ++i) {
        double c0 = u[id3(N, i, j, k)];
        double sum = 0.0;
        for (int ax = 0; ax < 3; ++ax) {
          int di = ax == 0, dj = ax == 1, dk = ax == 2;
          double m1 = value_at(u, N, i - di, j - dj, k - dk);
          double p1 = value_at(u, N, i + di, j + dj, k + dk);
          if (order == 2) {
            sum += (m1 - 2.0 * c0 + p1) / (h * h);
          } else {
            double m2 = value_at(u, N, i - 2 * di, j - 2 * dj, k - 2 * dk);
            double p2 = value_at(u, N, i + 2 * di, j + 2 * dj, k + 2 * dk);
            sum += (-m2 + 16.0 * m1 - 30.0 * c0 + 16.0 * p1 - p2) / (12.0 * h * h);
          }
        }
        out[id3(N, i, j, k)] = sum;
      }
}

/* out = A u with A = W - c Delta_h: the matrix of one implicit-Euler
 * substep (Sec. 1.1, the sweep equation, implicit part); W = I except for
 * the compact stencil. */
void or_apply_A(int N, int order, double c, const double* u, double* out) {
  size_t n = n3(N);
  double* w = (double*)malloc(n * sizeof(double));
  or_weight(N, order, u, w);
  or_laplacian(N, order, u, out);
  #pragma omp parallel for
  for (size_t p = 0; p < n; ++p) out[p] = w[p] - c * out[p];
  free(w);
}

/* r = b - A u */
void or_residual(int N, int order, double c, const double* u, const double* b, double* r) {
  or_apply_A(N, order, c, u, r);
  size_t n = n3(N);
  #pragma omp parallel for
  for (size_t p = 0; p < n; ++p) r[p] = b[p] - r[p];
}

double or_maxabs(size_t n, const double* v) {
  double m = 0.0;
  for (size_t p = 0; p < n; ++p) {
    double a = fabs(v[p]);
    if (a > m || a != a) m = a;
  }
  return m;
}

/* ------------------------------------------------------------------------ */
/* Geometric multigrid (Sec. 1.2: multigrid solve of the implicit systems,   */
/* coarsest grid of one unknown)                                             */
/* ------------------------------------------------------------------------ */

/* Damping factors from local Fourier analysis of each stencil's Laplacian:
 * 2 / (smallest + largest high-frequency symbol of the Jacobi-normalised
 * operator); the compact operator's range is [1/2, 4/3]. */
static double jacobi_omega(int order) {
  if (order == OR_COMPACT) return 12.0 / 11.0;
  return order == 2 ? 6.0 / 7.0 : 9.0 / 11.0;
}

/* Diagonal used by the smoother: the constant interior diagonal of A. */
static double jacobi_diag(int N, int order, double c) {
  double h = 1.0 / (N + 1);
  if (order == OR_COMPACT) return 0.5 + c * 4.0 / (h * h);
  return order == 2 ? 1.0 + c * 6.0 / (h * h) : 1.0 + c * 90.0 / (12.0 * h * h);
}

/* out = u + omega D^{-1} (b - A u): one damped-Jacobi sweep. */
void or_jacobi(int N, int order, double c, const double* u, const double* b, double* out) {
  size_t n = n3(N);
  double* r = (double*)malloc(n * sizeof(double));
  or_residual(N, order, c, u, b, r);
  double w = jacobi_omega(order), d = jacobi_diag(N, order, c);
  #pragma omp parallel for
  for (size_t p = 0; p < n; ++p) out[p] = u[p] + w * r[p] / d;
  free(r);
}

/* Full weighting: coarse I <- sum over a,b,c in {-1,0,1} of
 * w_a w_b w_c r(2I+a, 2J+b, 2K+c), with w_0 = 1/2 and w_{+-1} = 1/4. */
void or_restrict_fw(int Nf, const double* r, double* bc) {
  int Nc = (Nf - 1) / 2;
  const double w[3] = {0.25, 0.5, 0.25};
  #pragma omp parallel for
  for (int K = 1; K <= Nc; ++K)
    for (int J = 1; J <= Nc; ++J)
      for (int I = 1; I <= Nc; ++I) {
        double s = 0.0;
        for (int c = -1; c <= 1; ++c)
          for (int b = -1; b <= 1; ++b)
            for (int a = -1; a <= 1; ++a)
              s += w[a + 1] * w[b + 1] * w[c + 1] * r[id3(Nf, 2 * I + a, 2 * J + b, 2 * K + c)];
        bc[id3(Nc, I, J, K)] = s;
      }
}

/* Coarse value with zero Dirichlet boundary, for interpolation. */
static double coarse_at(const double* e, int Nc, int I, int J, int K) {
  if (I < 1 || I > Nc || J < 1 || J > Nc || K < 1 || K > Nc) return 0.0;
  return e[id3(Nc, I, J, K)];
}

/* uf += P e: trilinear interpolation, fine 2I = coarse I, odd fine points
 * take the mean of the two coarse neighbours along every odd axis. */
void or_prolong_add(int Nc, const double* e, double* uf) {
  int Nf = 2 * Nc + 1;
  #pragma omp parallel for
  for (int k = 1; k <= Nf; ++k)
    for (int j = 1; j <= Nf; ++j)
      for (int i = 1; i <= Nf; ++i) {
        int ia[2], ja[2], ka[2], ni, nj, nk;
        if (i % 2 == 0) { ia[0] = i / 2; ni = 1; } else { ia[0] = (i - 1) / 2; ia[1] = (i + 1) / 2; ni = 2; }
        if (j % 2 == 0) { ja[0] = j / 2; nj = 1; } else { ja[0] = (j - 1) / 2; ja[1] = (j + 1) / 2; nj = 2; }
        if (k % 2 == 0) { ka[0] = k / 2; nk = 1; } else { ka[0] = (k - 1) / 2; ka[1] = (k + 1) / 2; nk = 2; }
        double s = 0.0;
        for (int c = 0; c < nk; ++c)
          for (int b = 0; b < nj; ++b)
            for (int a = 0; a < ni; ++a)
              s += coarse_at(e, Nc, ia[a], ja[b], ka[c]) / (double)(ni * nj * nk);
        uf[id3(Nf, i, j, k)] += s;
      }
}

/* One axis of the cubic interpolation: value at fine index i (1..2Nc+1) from
 * the coarse line e(1..Nc) with zero boundary values and odd reflection
 * beyond them: even i take the coarse value, odd i the 4-point Lagrange
 * midpoint (-e(I-1) + 9 e(I) + 9 e(I+1) - e(I+2)) / 16. */
static double cubic_line_at(const double* e, int stride, int Nc, int i) {
  if (i % 2 == 0) return e[(size_t)(i / 2 - 1) * stride];
  int I = (i - 1) / 2;
  double v[4];
  for (int q = 0; q < 4; ++q) {
    int a = I - 1 + q;
    double sgn = 1.0;
    if (a == 0 || a == Nc + 1) { v[q] = 0.0; continue; }
    if (a < 0) { a = -a; sgn = -1.0; }
    if (a > Nc + 1) { a = 2 * (Nc + 1) - a; sgn = -1.0; }
    v[q] = sgn * e[(size_t)(a - 1) * stride];
  }
  return (-v[0] + 9.0 * v[1] + 9.0 * v[2] - v[3]) / 16.0;
}

/* Weight of point q (0..npts-1) of the npts-point Lagrange rule on equally
 * spaced points, evaluated halfway between the middle two: with the points at
 * X_q / 2, X_q = 2q - (npts - 1) (odd integers), the weight is the product
 * over r != q of (0 - X_r) / (X_q - X_r), formed in integers and divided once
 * (npts = 4 gives (-1, 9, 9, -1) / 16). */
static double lagrange_mid_weight(int npts, int q) {
  long long num = 1, den = 1;
  for (int r = 0; r < npts; ++r) {
    if (r == q) continue;
    long long xr = 2 * r - (npts - 1), xq = 2 * q - (npts - 1);
    num *= -xr;
    den *= xq - xr;
  }
  return (double)num / (double)den;
}

/* Coarse line value at coarse index a (any integer) of the odd extension
 * about both boundary points (0 and Nc + 1, where the value is zero): period
 * 2 (Nc + 1), odd about 0. */
static double odd_ext_at(const double* e, int stride, int Nc, int a) {
  int per = 2 * (Nc + 1);
  int r = ((a % per) + per) % per;
  if (r == 0 || r == Nc + 1) return 0.0;
  if (r > Nc + 1) return -e[(size_t)(per - r - 1) * stride];
  return e[(size_t)(r - 1) * stride];
}

/* One axis of the npts-point (npts = 6 or 8) midpoint rule: even fine
 * indices take the coarse value, odd ones sum the weighted npts coarse values
 * centred on the midpoint, in order of the points, on the odd extension. */
static double lagrange_line_at(const double* e, int stride, int Nc, int i, int npts) {
  if (i % 2 == 0) return e[(size_t)(i / 2 - 1) * stride];
  int I = (i - 1) / 2; /* the midpoint lies between coarse I and I + 1 */
  double s = 0.0;
  for (int q = 0; q < npts; ++q)
    s += lagrange_mid_weight(npts, q) * odd_ext_at(e, stride, Nc, I - npts / 2 + 1 + q);
  return s;
}

static double line_at(const double* e, int stride, int Nc, int i, int npts) {
  return npts == 4 ? cubic_line_at(e, stride, Nc, i) : lagrange_line_at(e, stride, Nc, i, npts);
}

/* uf += P e: tensor-product npts-point midpoint interpolation (npts = 4:
 * cubic, 6, 8), x, then y, then z. */
void or_prolong_add_lagrange(int Nc, int npts, const double* e, double* uf) {
  int Nf = 2 * Nc + 1;
  double* tx = (double*)malloc((size_t)Nf * Nc * Nc * sizeof(double));
  double* txy = (double*)malloc((size_t)Nf * Nf * Nc * sizeof(double));
  #pragma omp parallel for
  for (int K = 0; K < Nc; ++K)
    for (int J = 0; J < Nc; ++J)
      for (int i = 1; i <= Nf; ++i)
        tx[((size_t)K * Nc + J) * Nf + (i - 1)] =
            line_at(e + ((size_t)K * Nc + J) * Nc, 1, Nc, i, npts);
  #pragma omp parallel for
  for (int K = 0; K < Nc; ++K)
    for (int j = 1; j <= Nf; ++j)
      for (int i = 0; i < Nf; ++i)
        txy[((size_t)K * Nf + (j - 1)) * Nf + i] =
            line_at(tx + (size_t)K * Nc * Nf + i, Nf, Nc, j, npts);
  #pragma omp parallel for
  for (int k = 1; k <= Nf; ++k)
    for (int j = 0; j < Nf; ++j)
      for (int i = 0; i < Nf; ++i)
        uf[((size_t)(k - 1) * Nf + j) * Nf + i] += line_at(txy + (size_t)j * Nf + i, Nf * Nf, Nc, k, npts);
  free(tx); free(txy);
}

/* uf += P3 e: tensor-product cubic interpolation, x, then y, then z. */
void or_prolong_add_cubic(int Nc, const double* e, double* uf) {
  or_prolong_add_lagrange(Nc, 4, e, uf);
}

/* Exact solve on the one-unknown grid: A11 is read off by applying A to the
 * unit field. */
static void solve_one_unknown(int order, double c, double* u, const double* b) {
  double one = 1.0, a11 = 0.0;
  or_apply_A(1, order, c, &one, &a11);
  u[0] = b[0] / a11;
}

/* One V(nu1, nu2) cycle for A u = b, u updated in place. */
void or_vcycle(int N, int order, double c, double* u, const double* b, int nu1, int nu2) {
  if (N == 1) { solve_one_unknown(order, c, u, b); return; }
  size_t n = n3(N);
  double* t = (double*)malloc(n * sizeof(double));
  for (int s = 0; s < nu1; ++s) { or_jacobi(N, order, c, u, b, t); memcpy(u, t, n * sizeof(double)); }
  or_residual(N, order, c, u, b, t);
  int Nc = (N - 1) / 2;
  size_t nc = n3(Nc);
  double* bc = (double*)malloc(nc * sizeof(double));
  double* uc = (double*)calloc(nc, sizeof(double));
  or_restrict_fw(N, t, bc);
  or_vcycle(Nc, order, c, uc, bc, nu1, nu2);
  or_prolong_add(Nc, uc, u);
  for (int s = 0; s < nu2; ++s) { or_jacobi(N, order, c, u, b, t); memcpy(u, t, n * sizeof(double)); }
  free(bc); free(uc); free(t);
}

static int mg_levels_ok(int N) {
  int n = N;
  while (n > 1) { if (n % 2 == 0) return 0; n = (n - 1) / 2; }
  return n == 1;
}

/* Solve (W - c Delta_h) u = b, warm-started from u.  tol >= 0: cycle while
 * max|b - A u| > tol, at most max_cycles; tol < 0: exactly max_cycles. */
int or_mg_solve(int N, int order, double c, double* u, const double* b, double tol,
                int max_cycles, int nu1, int nu2, int* cycles_out, double* res_out) {
  if (!mg_levels_ok(N)) return OR_EINVAL;
  size_t n = n3(N);
  double* r = (double*)malloc(n * sizeof(double));
  or_residual(N, order, c, u, b, r);
  double res = or_maxabs(n, r);
  int cycles = 0;
  while (cycles < max_cycles && (tol < 0 || res > tol)) {
    or_vcycle(N, order, c, u, b, nu1, nu2);
    ++cycles;
    or_residual(N, order, c, u, b, r);
    res = or_maxabs(n, r);
  }
  free(r);
  if (cycles_out) *cycles_out = cycles;
  if (res_out) *res_out = res;
  return (tol >= 0 && res > tol) ? OR_ENOTCONV : OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Collocation: Gauss-Lobatto nodes and the integration matrices Q and S     */
/* (Sec. 1.1, the collocation formula and the spectral quadrature)          */
/* ------------------------------------------------------------------------ */

/* Gauss-Lobatto nodes on [0, 1]: the end points and the roots of P'_{M-1}
 * mapped from [-1, 1]. */
int or_gl_nodes(int M, double* tau) {
  switch (M) {
    case 2: tau[0] = 0.0; tau[1] = 1.0; return OR_OK;
    case 3: tau[0] = 0.0; tau[1] = 0.5; tau[2] = 1.0; return OR_OK;
    case 4:
      tau[0] = 0.0; tau[1] = 0.5 * (1.0 - 1.0 / sqrt(5.0));
      tau[2] = 0.5 * (1.0 + 1.0 / sqrt(5.0)); tau[3] = 1.0; return OR_OK;
    case 5:
      tau[0] = 0.0; tau[1] = 0.5 * (1.0 - sqrt(3.0 / 7.0)); tau[2] = 0.5;
      tau[3] = 0.5 * (1.0 + sqrt(3.0 / 7.0)); tau[4] = 1.0; return OR_OK;
    default: return OR_EINVAL;
  }
}

/* Monomial coefficients a[0..M-1] of the Lagrange basis polynomial l_j. */
static void lagrange_coeffs(int M, const double* tau, int j, double* a) {
  for (int p = 0; p < M; ++p) a[p] = 0.0;
  a[0] = 1.0;
  int deg = 0;
  for (int i = 0; i < M; ++i) {
    if (i == j) continue;
    double den = tau[j] - tau[i];
    /* multiply the polynomial by (s - tau_i) / den */
    for (int p = deg + 1; p >= 0; --p) {
      double hi = p > 0 ? a[p - 1] : 0.0;
      double lo = p <= deg ? a[p] : 0.0;
      a[p] = (hi - tau[i] * lo) / den;
    }
    ++deg;
  }
}

/* Q[m][j] = integral from 0 to tau_m of l_j(s) ds (step length 1). */
int or_qmatrix(int M, double* Q) {
  double tau[8], a[8];
  if (or_gl_nodes(M, tau) != OR_OK) return OR_EINVAL;
  for (int j = 0; j < M; ++j) {
    lagrange_coeffs(M, tau, j, a);
    for (int m = 0; m < M; ++m) {
      double s = 0.0, tp = tau[m];
      for (int p = 0; p < M; ++p) { s += a[p] * tp / (p + 1); tp *= tau[m]; }
      Q[m * M + j] = s;
    }
  }
  return OR_OK;
}

/* S[m][j] = Q[m+1][j] - Q[m][j], m = 0..M-2: node-to-node integrals. */
int or_smatrix(int M, double* S) {
  double Q[64];
  if (or_qmatrix(M, Q) != OR_OK) return OR_EINVAL;
  for (int m = 0; m + 1 < M; ++m)
    for (int j = 0; j < M; ++j) S[m * M + j] = Q[(m + 1) * M + j] - Q[m * M + j];
  return OR_OK;
}

/* l_m(s) for the nodes tau (Lagrange basis value). */
static double lagrange_value(int M, const double* tau, int m, double s) {
  double v = 1.0;
  for (int i = 0; i < M; ++i)
    if (i != m) v *= (s - tau[i]) / (tau[m] - tau[i]);
  return v;
}

/* ------------------------------------------------------------------------ */
/* Problem data (Sec. 1, Eqs. 3-4)                                           */
/* ------------------------------------------------------------------------ */

/* Phi(x) = sin(pi x1) sin(pi x2) sin(pi x3) at the interior points. */
void or_phi(int N, double* phi) {
  double h = 1.0 / (N + 1);
  #pragma omp parallel for
  for (int k = 1; k <= N; ++k)
    for (int j = 1; j <= N; ++j)
      for (int i = 1; i <= N; ++i)
        phi[id3(N, i, j, k)] = sin(OR_PI * i * h) * sin(OR_PI * j * h) * sin(OR_PI * k * h);
}

/* Time factor g of the forcing f = Phi(x) g(t), Eq. 3 with the coefficient
 * kappa in front of nu pi^2 (kappa = 1 as printed). */
static double forcing_g(const or_problem* P, double t) {
  if (!P->forcing) return 0.0;
  return -(sin(t) - P->kappa * P->nu * OR_PI * OR_PI * cos(t));
}

/* ------------------------------------------------------------------------ */
/* SDC (Sec. 1.1: IMEX-Euler sweep, spectral quadrature, residual)           */
/* ------------------------------------------------------------------------ */

/* F = f^I(U) = nu Delta_h U at one node. */
static void eval_fI(const or_level* L, const or_problem* P, const double* u, double* F) {
  or_laplacian(L->N, L->order, u, F);
  size_t n = n3(L->N);
  #pragma omp parallel for
  for (size_t p = 0; p < n; ++p) F[p] = P->nu * F[p];
}

/* Recompute F at every node from U (U and F hold M fields of N^3). */
void or_eval_F_all(const or_level* L, const or_problem* P, const double* U, double* F) {
  size_t n = n3(L->N);
  for (int m = 0; m < L->M; ++m) eval_fI(L, P, U + m * n, F + m * n);
}

/* Spread the initial value u0 to all M nodes (initial SDC iterate). */
void or_spread(const or_level* L, const or_problem* P, const double* u0, double* U, double* F) {
  size_t n = n3(L->N);
  for (int m = 0; m < L->M; ++m) memcpy(U + m * n, u0, n * sizeof(double));
  or_eval_F_all(L, P, U, F);
}

double or_sdc_residual(const or_level* L, const or_problem* P, double t0, double dt,
                       const double* U, const double* F, const double* tauQ);

/* One IMEX-Euler SDC sweep over [t0, t0 + dt] (the sweep equation of
 * Sec. 1.1), U and F updated in place; for the compact stencil in the
 * weighted form (W - dt_m nu L) U_{m+1} = W U_m - dt_m F_{m+1} + quadrature.  tauQ (M fields or NULL) is the FAS
 * correction in cumulative form; the sweep adds tauQ_{m+1} - tauQ_m on the
 * substep m.  The explicit part is the forcing, so its difference term is
 * evaluated as written and is zero. */
int or_sdc_sweep(const or_level* L, const or_problem* P, double t0, double dt, double* U,
                 double* F, const double* tauQ, or_stats* st) {
  int N = L->N, M = L->M, status = OR_OK;
  size_t n = n3(N);
  double tau[8], S[64];
  if (or_gl_nodes(M, tau) != OR_OK || or_smatrix(M, S) != OR_OK) return OR_EINVAL;
  /* Inner tolerance of this sweep's solves: fixed, or tied to the collocation
   * residual of the incoming iterate (the paper leaves the solver tolerance
   * open; the residual threshold applies to the outer iteration). */
  double mg_tol = P->mg_tol;
  if (P->mg_rel > 0 && P->mg_tol >= 0) {
    double r_in = or_sdc_residual(L, P, t0, dt, U, F, tauQ);
    if (P->mg_rel * r_in > mg_tol) mg_tol = P->mg_rel * r_in;
  }
  double* Fold = (double*)malloc((size_t)M * n * sizeof(double));
  double* phi = (double*)malloc(n * sizeof(double));
  double* wphi = (double*)malloc(n * sizeof(double));
  double* wu = (double*)malloc(n * sizeof(double));
  double* rhs = (double*)malloc(n * sizeof(double));
  memcpy(Fold, F, (size_t)M * n * sizeof(double));
  or_phi(N, phi);
  /* the weighted form W U' = F + W f (W = I but for the compact stencil) */
  or_weight(N, L->order, phi, wphi);
  for (int m = 0; m + 1 < M; ++m) {
    double tm = t0 + dt * tau[m], tm1 = t0 + dt * tau[m + 1];
    double dtm = dt * (tau[m + 1] - tau[m]);
    or_weight(N, L->order, U + m * n, wu);
    #pragma omp parallel for
    for (size_t p = 0; p < n; ++p) {
      double fe_new = wphi[p] * forcing_g(P, tm); /* W f^E(U^{k+1}_m, t_m) */
      double fe_old = wphi[p] * forcing_g(P, tm); /* W f^E(U^k_m, t_m) */
      double quad = 0.0;
      for (int j = 0; j < M; ++j)
        quad += S[m * M + j] * (Fold[j * n + p] + wphi[p] * forcing_g(P, t0 + dt * tau[j]));
      double v = wu[p] + dtm * (fe_new - fe_old) - dtm * Fold[(m + 1) * n + p] + dt * quad;
      if (tauQ) v += tauQ[(m + 1) * n + p] - tauQ[m * n + p];
      rhs[p] = v;
    }
    (void)tm1;
    int cyc = 0;
    double res = 0.0;
    int rc = or_mg_solve(N, L->order, dtm * P->nu, U + (m + 1) * n, rhs, mg_tol, P->mg_max,
                         P->nu1, P->nu2, &cyc, &res);
    if (rc == OR_ENOTCONV) { status = OR_ENOTCONV; if (st) st->notconv++; }
    else if (rc != OR_OK) { status = rc; break; }
    if (st) { st->vcycles += cyc; st->solves += 1; st->vcycle_points += (double)cyc * n3(N); }
    eval_fI(L, P, U + (m + 1) * n, F + (m + 1) * n);
  }
  if (st) st->sweeps += 1;
  free(Fold); free(phi); free(wphi); free(wu); free(rhs);
  return status;
}

/* Collocation residual max_m max_x |W U_0 + dt sum_j Q_{m,j} (F_j + W f^E_j)
 * + tauQ_m - W U_m| over the nodes m = 1..M-1 (W = I but for the compact
 * stencil, whose residual is taken in the weighted form). */
double or_sdc_residual(const or_level* L, const or_problem* P, double t0, double dt,
                       const double* U, const double* F, const double* tauQ) {
  int N = L->N, M = L->M;
  size_t n = n3(N);
  double tau[8], Q[64];
  or_gl_nodes(M, tau);
  or_qmatrix(M, Q);
  double* phi = (double*)malloc(n * sizeof(double));
  double* wphi = (double*)malloc(n * sizeof(double));
  double* wu = (double*)malloc((size_t)M * n * sizeof(double));
  or_phi(N, phi);
  or_weight(N, L->order, phi, wphi);
  for (int m = 0; m < M; ++m) or_weight(N, L->order, U + m * n, wu + m * n);
  double res = 0.0;
  for (int m = 1; m < M; ++m)
    for (size_t p = 0; p < n; ++p) {
      double quad = 0.0;
      for (int j = 0; j < M; ++j)
        quad += Q[m * M + j] * (F[j * n + p] + wphi[p] * forcing_g(P, t0 + dt * tau[j]));
      double v = wu[p] + dt * quad - wu[m * n + p];
      if (tauQ) v += tauQ[m * n + p];
      double a = fabs(v);
      if (a > res || a != a) res = a;
    }
  free(phi); free(wphi); free(wu);
  return res;
}

/* Serial single-level SDC over nsteps steps of size dt: every step spreads
 * its initial value, then sweeps nsweeps times (tol < 0), or until the
 * residual is <= tol (at most nsweeps). */
int or_sdc_run(const or_level* L, const or_problem* P, double dt, int nsteps, int nsweeps,
               double tol, const double* u0, double* uT, or_stats* st) {
  int N = L->N, M = L->M, status = OR_OK;
  size_t n = n3(N);
  double* U = (double*)malloc((size_t)M * n * sizeof(double));
  double* F = (double*)malloc((size_t)M * n * sizeof(double));
  double* ucur = (double*)malloc(n * sizeof(double));
  memcpy(ucur, u0, n * sizeof(double));
  for (int s = 0; s < nsteps; ++s) {
    double t0 = s * dt;
    or_spread(L, P, ucur, U, F);
    for (int k = 0; k < nsweeps; ++k) {
      if (tol >= 0) {
        double r = or_sdc_residual(L, P, t0, dt, U, F, NULL);
        if (st) st->residual = r;
        if (r <= tol) break;
      }
      int rc = or_sdc_sweep(L, P, t0, dt, U, F, NULL, st);
      if (rc == OR_ENOTCONV) status = rc;
      else if (rc != OR_OK) { status = rc; goto done; }
    }
    if (st) st->residual = or_sdc_residual(L, P, t0, dt, U, F, NULL);
    memcpy(ucur, U + (size_t)(M - 1) * n, n * sizeof(double));
  }
  memcpy(uT, ucur, n * sizeof(double));
done:
  free(U); free(F); free(ucur);
  return status;
}

/* ------------------------------------------------------------------------ */
/* FAS coupling of two levels (Sec. 1.1: MLSDC / PFASST with coarsening in   */
/* nodes, mesh and stencil order)                                            */
/* ------------------------------------------------------------------------ */

/* Fine node matching coarse node m (nested Gauss-Lobatto sets), or -1. */
static int node_map(int MF, int MG, int m) {
  double tf[8], tg[8];
  or_gl_nodes(MF, tf);
  or_gl_nodes(MG, tg);
  for (int j = 0; j < MF; ++j)
    if (fabs(tf[j] - tg[m]) < 1e-14) return j;
  return -1;
}

static int fas_check(const or_level* F, const or_level* G) {
  if (!(F->N == G->N || F->N == 2 * G->N + 1)) return OR_EINVAL;
  if (G->order == OR_COMPACT) return OR_EINVAL; /* compact: fine level only */
  double tf[8], tg[8];
  if (or_gl_nodes(F->M, tf) || or_gl_nodes(G->M, tg)) return OR_EINVAL;
  for (int m = 0; m < G->M; ++m)
    if (node_map(F->M, G->M, m) < 0) return OR_EINVAL;
  return OR_OK;
}

/* Injection in space: coarse I <- fine 2I (or the identity for equal N). */
static void inject(int NF, int NG, const double* uf, double* ug) {
  if (NF == NG) { memcpy(ug, uf, n3(NF) * sizeof(double)); return; }
  for (int K = 1; K <= NG; ++K)
    for (int J = 1; J <= NG; ++J)
      for (int I = 1; I <= NG; ++I) ug[id3(NG, I, J, K)] = uf[id3(NF, 2 * I, 2 * J, 2 * K)];
}

/* Restriction of the fine state to the coarse level and the FAS correction
 * in cumulative (Q) form:
 *   U^G_m = R U^F_{j(m)},  F^G_m = nu Delta^G U^G_m,
 *   tauQ_m = R(dt sum_j Q^F_{j(m),j} (F^F_j + f^E_j)) - dt sum_i Q^G_{m,i} (F^G_i + f^E_i).
 * A compact fine level integrates the weighted system, so its integral is
 * mapped back by W^{-1} before the injection (Sec. 1.2, the weighting-matrix
 * inversion for the FAS correction), in the equivalent form
 * U_j - U_0 + W^{-1} r: a multigrid solve of W x = r (c = 0), warm-started
 * from r, to max|r - W x| <= max(mg_tol, OR_W_REL max|r|); node 0, whose
 * integral is zero, is not solved.
 * UGr receives a copy of the restricted U^G for the later correction. */
int or_fas_restrict_st(const or_level* LF, const or_level* LG, const or_problem* P, double t0,
                       double dt, const double* UF, const double* FF, double* UG, double* FG,
                       double* UGr, double* tauQ, or_stats* st) {
  if (fas_check(LF, LG) != OR_OK) return OR_EINVAL;
  int status = OR_OK;
  int NF = LF->N, NG = LG->N, MF = LF->M, MG = LG->M;
  size_t nf = n3(NF), ng = n3(NG);
  double tf[8], tg[8], QF[64], QG[64];
  or_gl_nodes(MF, tf); or_gl_nodes(MG, tg); or_qmatrix(MF, QF); or_qmatrix(MG, QG);
  double* phif = (double*)malloc(nf * sizeof(double));
  double* phig = (double*)malloc(ng * sizeof(double));
  double* tmpf = (double*)malloc(nf * sizeof(double));
  double* xf = (double*)malloc(nf * sizeof(double));
  double* tmpg = (double*)malloc(ng * sizeof(double));
  or_phi(NF, phif); or_phi(NG, phig);
  if (LF->order == OR_COMPACT) {
    or_weight(NF, LF->order, phif, xf);
    memcpy(phif, xf, nf * sizeof(double)); /* W f^E = g(t) W Phi on the fine level */
  }
  for (int m = 0; m < MG; ++m) {
    int jm = node_map(MF, MG, m);
    inject(NF, NG, UF + (size_t)jm * nf, UG + (size_t)m * ng);
  }
  memcpy(UGr, UG, (size_t)MG * ng * sizeof(double));
  or_eval_F_all(LG, P, UG, FG);
  for (int m = 0; m < MG; ++m) {
    int jm = node_map(MF, MG, m);
    #pragma omp parallel for
    for (size_t p = 0; p < nf; ++p) {
      double q = 0.0;
      for (int j = 0; j < MF; ++j)
        q += QF[jm * MF + j] * (FF[(size_t)j * nf + p] + phif[p] * forcing_g(P, t0 + dt * tf[j]));
      tmpf[p] = dt * q;
    }
    if (LF->order == OR_COMPACT && jm != 0) {
      /* W^{-1} (integral) = U_jm - U_0 + W^{-1} r with the weighted residual
       * r = W U_0 + integral - W U_jm: only r goes through the solver, so an
       * inexact solve changes the correction but not the fixed point. */
      double* wu0 = (double*)malloc(nf * sizeof(double));
      double* wuj = (double*)malloc(nf * sizeof(double));
      or_weight(NF, LF->order, UF, wu0);
      or_weight(NF, LF->order, UF + (size_t)jm * nf, wuj);
      for (size_t p = 0; p < nf; ++p) tmpf[p] = wu0[p] + tmpf[p] - wuj[p];
      double rmax = or_maxabs(nf, tmpf);
      double wtol = P->mg_tol;
      if (P->mg_tol >= 0 && OR_W_REL * rmax > wtol) wtol = OR_W_REL * rmax;
      int cyc = 0;
      double res = 0.0;
      memcpy(xf, tmpf, nf * sizeof(double));
      int rc = or_mg_solve(NF, LF->order, 0.0, xf, tmpf, wtol, P->mg_max, P->nu1, P->nu2,
                           &cyc, &res);
      if (rc == OR_ENOTCONV) { status = rc; if (st) st->notconv++; }
      else if (rc != OR_OK) { status = rc; free(wu0); free(wuj); break; }
      if (st) { st->vcycles += cyc; st->solves += 1; st->vcycle_points += (double)cyc * nf; }
      for (size_t p = 0; p < nf; ++p) tmpf[p] = UF[(size_t)jm * nf + p] - UF[p] + xf[p];
      free(wu0); free(wuj);
    }
    inject(NF, NG, tmpf, tmpg);
    #pragma omp parallel for
    for (size_t p = 0; p < ng; ++p) {
      double q = 0.0;
      for (int i = 0; i < MG; ++i)
        q += QG[m * MG + i] * (FG[(size_t)i * ng + p] + phig[p] * forcing_g(P, t0 + dt * tg[i]));
      tauQ[(size_t)m * ng + p] = tmpg[p] - dt * q;
    }
  }
  free(phif); free(phig); free(tmpf); free(xf); free(tmpg);
  return status;
}

int or_fas_restrict(const or_level* LF, const or_level* LG, const or_problem* P, double t0,
                    double dt, const double* UF, const double* FF, double* UG, double* FG,
                    double* UGr, double* tauQ) {
  return or_fas_restrict_st(LF, LG, P, t0, dt, UF, FF, UG, FG, UGr, tauQ, NULL);
}

/* Coarse-to-fine correction: Delta_m = U^G_m - UGr_m at the coarse nodes,
 * Lagrange interpolation in time to every fine node, trilinear (or the
 * interp-point midpoint rule) in space, U^F_j += that, then F^F is recomputed
 * from the new U^F. */
int or_fas_interpolate(const or_level* LF, const or_level* LG, const or_problem* P,
                       const double* UG, const double* UGr, double* UF, double* FF) {
  if (fas_check(LF, LG) != OR_OK) return OR_EINVAL;
  int NF = LF->N, NG = LG->N, MF = LF->M, MG = LG->M;
  size_t nf = n3(NF), ng = n3(NG);
  double tf[8], tg[8];
  or_gl_nodes(MF, tf); or_gl_nodes(MG, tg);
  double* d = (double*)malloc(ng * sizeof(double));
  for (int j = 0; j < MF; ++j) {
    #pragma omp parallel for
    for (size_t p = 0; p < ng; ++p) {
      double s = 0.0;
      for (int m = 0; m < MG; ++m)
        s += lagrange_value(MG, tg, m, tf[j]) * (UG[(size_t)m * ng + p] - UGr[(size_t)m * ng + p]);
      d[p] = s;
    }
    if (NF == NG) {
      for (size_t p = 0; p < nf; ++p) UF[(size_t)j * nf + p] += d[p];
    } else if (P->interp == 4 || P->interp == 6 || P->interp == 8) {
      or_prolong_add_lagrange(NG, P->interp, d, UF + (size_t)j * nf);
    } else {
      or_prolong_add(NG, d, UF + (size_t)j * nf);
    }
  }
  free(d);
  or_eval_F_all(LF, P, UF, FF);
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Two-level MLSDC and the serial emulation of PFASST (Sec. 1.1)            */
/* ------------------------------------------------------------------------ */

typedef struct {
  int nsweeps_fine;   /* fine sweeps per iteration */
  int nsweeps_coarse; /* coarse sweeps per iteration and in the predictor */
  int max_iters;      /* iteration cap (exact count when tol < 0) */
  double tol;         /* fine collocation residual threshold */
  int predictor;      /* 1: coarse predictor before the first iteration */
} or_mlsdc_opts;

/* Coarse sweeps of one coarse state with its FAS correction. */
static int coarse_sweeps(const or_level* LG, const or_problem* P, double t0, double dt, double* UG,
                         double* FG, const double* tauQ, int nsw, or_stats* st) {
  int status = OR_OK;
  for (int s = 0; s < nsw; ++s) {
    int rc = or_sdc_sweep(LG, P, t0, dt, UG, FG, tauQ, st);
    if (rc == OR_ENOTCONV) status = rc;
    else if (rc != OR_OK) return rc;
  }
  return status;
}

/* Serial two-level MLSDC over nsteps steps.  Each step: spread the initial
 * value; optional predictor (restrict, coarse sweeps, interpolate); then
 * iterations of [fine sweeps, restrict + FAS, coarse sweeps, interpolate],
 * stopping when the fine residual is <= tol (or after max_iters). */
int or_mlsdc_run(const or_level* LF, const or_level* LG, const or_problem* P, double dt,
                 int nsteps, const or_mlsdc_opts* o, const double* u0, double* uT,
                 or_stats* st) {
  if (fas_check(LF, LG) != OR_OK) return OR_EINVAL;
  int MF = LF->M, MG = LG->M, status = OR_OK;
  size_t nf = n3(LF->N), ng = n3(LG->N);
  double* UF = (double*)malloc((size_t)MF * nf * sizeof(double));
  double* FF = (double*)malloc((size_t)MF * nf * sizeof(double));
  double* UG = (double*)malloc((size_t)MG * ng * sizeof(double));
  double* FG = (double*)malloc((size_t)MG * ng * sizeof(double));
  double* UGr = (double*)malloc((size_t)MG * ng * sizeof(double));
  double* tQ = (double*)malloc((size_t)MG * ng * sizeof(double));
  double* ucur = (double*)malloc(nf * sizeof(double));
  memcpy(ucur, u0, nf * sizeof(double));
  for (int s = 0; s < nsteps; ++s) {
    double t0 = s * dt;
    or_spread(LF, P, ucur, UF, FF);
    if (o->predictor) {
      if (or_fas_restrict_st(LF, LG, P, t0, dt, UF, FF, UG, FG, UGr, tQ, st) == OR_ENOTCONV)
        status = OR_ENOTCONV;
      int rc = coarse_sweeps(LG, P, t0, dt, UG, FG, tQ, o->nsweeps_coarse, st);
      if (rc != OR_OK && rc != OR_ENOTCONV) { status = rc; goto done; }
      if (rc == OR_ENOTCONV) status = rc;
      or_fas_interpolate(LF, LG, P, UG, UGr, UF, FF);
    }
    for (int it = 0; it < o->max_iters; ++it) {
      for (int k = 0; k < o->nsweeps_fine; ++k) {
        int rc = or_sdc_sweep(LF, P, t0, dt, UF, FF, NULL, st);
        if (rc != OR_OK && rc != OR_ENOTCONV) { status = rc; goto done; }
        if (rc == OR_ENOTCONV) status = rc;
      }
      if (or_fas_restrict_st(LF, LG, P, t0, dt, UF, FF, UG, FG, UGr, tQ, st) == OR_ENOTCONV)
        status = OR_ENOTCONV;
      int rc = coarse_sweeps(LG, P, t0, dt, UG, FG, tQ, o->nsweeps_coarse, st);
      if (rc != OR_OK && rc != OR_ENOTCONV) { status = rc; goto done; }
      if (rc == OR_ENOTCONV) status = rc;
      or_fas_interpolate(LF, LG, P, UG, UGr, UF, FF);
      if (st) st->iters += 1;
      double r = or_sdc_residual(LF, P, t0, dt, UF, FF, NULL);
      if (st) st->residual = r;
      if (o->tol >= 0 && r <= o->tol) break;
    }
    memcpy(ucur, UF + (size_t)(MF - 1) * nf, nf * sizeof(double));
  }
  memcpy(uT, ucur, nf * sizeof(double));
done:
  free(UF); free(FF); free(UG); free(FG); free(UGr); free(tQ); free(ucur);
  return status;
}

/* Serial emulation of two-level PFASST on blocks of nslices time slices.
 * Block start: the initial value is spread to every node of every slice.
 * Predictor: restrict all slices; coarse sweeps slice by slice, each slice
 * starting from the previous slice's coarse end value; interpolate; forward
 * the fine end values.  Iteration: fine sweeps on every slice; restrict all;
 * the same serial coarse pass; interpolate; forward fine end values
 * (U^F[p][0] <- U^F[p-1][M-1]); residual = max over slices.  Stops when the
 * residual is <= tol (or after max_iters).  slice_res (nslices values or
 * NULL) receives the last per-slice residuals; slice_nodes (nslices x M
 * fields of N^3, or NULL) the fine node values U^F[p][m] of the last block. */
int or_pfasst_run(const or_level* LF, const or_level* LG, const or_problem* P, double dt,
                  int nsteps, int nslices, const or_mlsdc_opts* o, const double* u0,
                  double* uT, double* slice_res, double* slice_nodes, or_stats* st) {
  if (fas_check(LF, LG) != OR_OK || nslices < 1 || nsteps % nslices != 0) return OR_EINVAL;
  int MF = LF->M, MG = LG->M, PS = nslices, status = OR_OK;
  size_t nf = n3(LF->N), ng = n3(LG->N);
  size_t sf = (size_t)MF * nf, sg = (size_t)MG * ng;
  double* UF = (double*)malloc(PS * sf * sizeof(double));
  double* FF = (double*)malloc(PS * sf * sizeof(double));
  double* UG = (double*)malloc(PS * sg * sizeof(double));
  double* FG = (double*)malloc(PS * sg * sizeof(double));
  double* UGr = (double*)malloc(PS * sg * sizeof(double));
  double* tQ = (double*)malloc(PS * sg * sizeof(double));
  double* ucur = (double*)malloc(nf * sizeof(double));
  memcpy(ucur, u0, nf * sizeof(double));
  for (int blk = 0; blk < nsteps / PS; ++blk) {
    double tb = (double)blk * PS * dt;
    for (int p = 0; p < PS; ++p) or_spread(LF, P, ucur, UF + p * sf, FF + p * sf);
    for (int it = -1; it < o->max_iters; ++it) {
      int predict = it < 0;
      if (predict && !o->predictor) continue;
      if (!predict)
        for (int p = 0; p < PS; ++p)
          for (int k = 0; k < o->nsweeps_fine; ++k) {
            int rc = or_sdc_sweep(LF, P, tb + p * dt, dt, UF + p * sf, FF + p * sf, NULL, st);
            if (rc != OR_OK && rc != OR_ENOTCONV) { status = rc; goto done; }
            if (rc == OR_ENOTCONV) status = rc;
          }
      for (int p = 0; p < PS; ++p)
        if (or_fas_restrict_st(LF, LG, P, tb + p * dt, dt, UF + p * sf, FF + p * sf, UG + p * sg,
                               FG + p * sg, UGr + p * sg, tQ + p * sg, st) == OR_ENOTCONV)
          status = OR_ENOTCONV;
      for (int p = 0; p < PS; ++p) {
        if (p > 0) {
          memcpy(UG + p * sg, UG + (p - 1) * sg + (size_t)(MG - 1) * ng, ng * sizeof(double));
          or_laplacian(LG->N, LG->order, UG + p * sg, FG + p * sg);
          for (size_t q = 0; q < ng; ++q) FG[p * sg + q] *= P->nu;
        }
        int rc = coarse_sweeps(LG, P, tb + p * dt, dt, UG + p * sg, FG + p * sg, tQ + p * sg,
                               o->nsweeps_coarse, st);
        if (rc != OR_OK && rc != OR_ENOTCONV) { status = rc; goto done; }
        if (rc == OR_ENOTCONV) status = rc;
      }
      for (int p = 0; p < PS; ++p)
        or_fas_interpolate(LF, LG, P, UG + p * sg, UGr + p * sg, UF + p * sf, FF + p * sf);
      for (int p = PS - 1; p >= 1; --p) {
        memcpy(UF + p * sf, UF + (p - 1) * sf + (size_t)(MF - 1) * nf, nf * sizeof(double));
        or_laplacian(LF->N, LF->order, UF + p * sf, FF + p * sf);
        for (size_t q = 0; q < nf; ++q) FF[p * sf + q] *= P->nu;
      }
      if (predict) continue;
      if (st) st->iters += 1;
      double r = 0.0;
      for (int p = 0; p < PS; ++p) {
        double rp = or_sdc_residual(LF, P, tb + p * dt, dt, UF + p * sf, FF + p * sf, NULL);
        if (slice_res) slice_res[p] = rp;
        if (rp > r || rp != rp) r = rp;
      }
      if (st) st->residual = r;
      if (o->tol >= 0 && r <= o->tol) break;
    }
    memcpy(ucur, UF + (PS - 1) * sf + (size_t)(MF - 1) * nf, nf * sizeof(double));
    if (slice_nodes) memcpy(slice_nodes, UF, PS * sf * sizeof(double));
  }
  memcpy(uT, ucur, nf * sizeof(double));
done:
  free(UF); free(FF); free(UG); free(FG); free(UGr); free(tQ); free(ucur);
  return status;
}
