/*
 * fdtd_oracle.c -- FP64 CPU oracle for the time-reversible FDTD gradient.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code, header, table or constant generator with the CUDA path.
 *
 * What it computes (all in double precision, plain loops, OpenMP over z):
 *   - the normalised 3D Yee leapfrog with a convolutional PML (CPML,
 *     Roden & Gedney, cited in Sec. 1 of the paper) on a zero-padded grid;
 *   - the objective L = sum_n l_n(E^{n+1}, H^{n+1/2}) on a detector plane;
 *   - the exact discrete gradient dL/d(eps_r) by a stored-history adjoint
 *     (reverse-mode of the discrete forward, no time reversal);
 *   - the paper's method step by step (Sec. 2): record the fields on the
 *     interface slices between the simulation volume and the PML, compressed
 *     by reduced bit-width and by keeping every k-th step; then run the
 *     time-reversed simulation with those slices injected back (linear or
 *     cubic interpolation in time) together with the adjoint;
 *   - the method's single operations (half-steps, their inverses and
 *     transposes, the objective and its seed, one face's interface layer),
 *     exported for tests that run the method piece by piece.
 *
 * Discretisation (the paper assumes a standard FDTD and cites the textbook):
 *   E and Ht = eta0*H; Ex(i+1/2,j,k), Ey(i,j+1/2,k), Ez(i,j,k+1/2),
 *   Hx(i,j+1/2,k+1/2), Hy(i+1/2,j,k+1/2), Hz(i+1/2,j+1/2,k), all stored at
 *   cell index (i,j,k).  S = c dt / dx (Eq. 1 with C = 0.99 gives
 *   S = 0.99/sqrt(3)).  One step n -> n+1:
 *     Ht^{n+1/2} = Ht^{n-1/2} - S * curlE(E^n)           (forward differences)
 *     E^{n+1}    = E^n + (S/eps_r) * (curlH(Ht^{n+1/2}) - J^{n+1/2})
 *   Out-of-grid neighbours read as zero, so curlH is the transpose of curlE.
 *   Each derivative d_u becomes (1/kappa_u) d_u + psi_u in the CPML, with
 *   psi_u <- b_u psi_u + a_u d_u evaluated at the derivative's own position.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  int nx, ny, nz;          /* cells */
  int P;                   /* CPML thickness on all faces (0 = none) */
  int periodic;            /* 1: periodic wrap (requires P == 0), 0: zero padding */
  int n_steps;
  double S;                /* Courant number c*dt/dx */
  double dx;               /* metres */
  int pml_m;               /* polynomial grading order */
  double sigma_factor;     /* sigma_max = sigma_factor*(m+1)/(eta0*dx) */
  double kappa_max;
  double alpha_factor;     /* alpha_max*dt/eps0 = alpha_factor * 2*pi*f0*dt */
  int src_kind;            /* 0 none, 1 point, 2 Gaussian plane, 3 uniform plane (plane wave) */
  int src_comp;            /* 0..2 = Ex..Ez */
  int src_axis;            /* plane normal for kind 2 */
  int src_pos[3];
  double src_sigma[2];     /* Gaussian widths along (u, v) in cells */
  double lambda0, rel_bw, t0_over_tau, amplitude;
  int det_kind;            /* 1 |E|^2, 2 Poynting along the plane normal */
  int det_axis, det_index, det_lo[2], det_hi[2];
  int dlo[3], dhi[3];      /* design box, half-open */
  /* optional second detector (kind 0 = none), e.g. the input-side flux of a
   * transmission ratio; its objective is M = sum_n m_n */
  int det2_kind, det2_axis, det2_index, det2_lo[2], det2_hi[2];
} ocfg;

/* ------------------------------------------------------------ helpers ---- */

#define NF 18               /* Ex Ey Ez Hx Hy Hz, psi[0..11] */
#define OFF_E 0
#define OFF_H 3
#define OFF_PSI 6

static size_t ncell(const ocfg* c) { return (size_t)c->nx * c->ny * c->nz; }
static size_t idx(const ocfg* c, int i, int j, int k) {
  return ((size_t)k * c->ny + j) * c->nx + i;
}
static int dim(const ocfg* c, int a) { return a == 0 ? c->nx : (a == 1 ? c->ny : c->nz); }

/* Field value with the grid's boundary rule: zero outside, or periodic wrap. */
static double at(const ocfg* c, const double* f, int i, int j, int k) {
  if (c->periodic) {
    i = (i + c->nx) % c->nx; j = (j + c->ny) % c->ny; k = (k + c->nz) % c->nz;
    return f[idx(c, i, j, k)];
  }
  if (i < 0 || j < 0 || k < 0 || i >= c->nx || j >= c->ny || k >= c->nz) return 0.0;
  return f[idx(c, i, j, k)];
}

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void oracle_set_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* ----------------------------------------------------- CPML profiles ----
 * Depth d in (0, 1] into the absorbing layer, measured from the interface at
 * the derivative's own position.  The lossless region is x in [P, N-P-1/2]:
 * it holds every E position (integer i) and every H position (i + 1/2) of the
 * interior cells [P, N-P).  Hence on the low side d = (P - x)/P, on the high
 * side d = (x - (N-P-1/2))/P, and d = 0 (no absorption) elsewhere.
 *   sigma~ = sigma*dt/eps0 = sigma_factor*(m+1)*S * d^m
 *   kappa  = 1 + (kappa_max - 1) d^m
 *   alpha~ = alpha_factor * 2*pi*f0*dt * (1 - d)
 *   b = exp(-(sigma~/kappa + alpha~)),  a = sigma~/(sigma~ kappa + kappa^2 alpha~) (b - 1)
 * Outside the layer b = a = 0 and 1/kappa = 1.
 */
static double depth(int N, int P, double x) {
  if (P <= 0) return 0.0;
  if (x < (double)P) return ((double)P - x) / P;
  double hi = (double)(N - P) - 0.5;
  if (x > hi) return (x - hi) / P;
  return 0.0;
}

static void profile_point(const ocfg* c, double d, double* b, double* a, double* kinv) {
  if (d <= 0.0) { *b = 0.0; *a = 0.0; *kinv = 1.0; return; }
  double m = (double)c->pml_m;
  double sig = c->sigma_factor * (m + 1.0) * c->S * pow(d, m);
  double kap = 1.0 + (c->kappa_max - 1.0) * pow(d, m);
  double f0dt = c->S * c->dx / c->lambda0;           /* f0*dt = (c/lambda0)*(S dx/c) */
  double alp = c->alpha_factor * 2.0 * M_PI * f0dt * (1.0 - d);
  *b = exp(-(sig / kap + alp));
  double den = sig * kap + kap * kap * alp;
  *a = den > 0.0 ? sig / den * (*b - 1.0) : 0.0;
  *kinv = 1.0 / kap;
}

/* out: 6 arrays of length N: b_E, a_E, kinv_E (integer positions),
 *      b_H, a_H, kinv_H (half-integer positions i + 1/2). */
int oracle_profiles(const ocfg* c, int axis, double* out) {
  int N = dim(c, axis);
  for (int i = 0; i < N; ++i) {
    profile_point(c, depth(N, c->P, (double)i), &out[0 * N + i], &out[1 * N + i], &out[2 * N + i]);
    profile_point(c, depth(N, c->P, i + 0.5), &out[3 * N + i], &out[4 * N + i], &out[5 * N + i]);
  }
  return 0;
}

typedef struct {
  double *be[3], *ae[3], *ke[3], *bh[3], *ah[3], *kh[3];
  double* store;
} oprof;

static int prof_alloc(const ocfg* c, oprof* p) {
  size_t tot = 6 * (size_t)(c->nx + c->ny + c->nz);
  p->store = (double*)malloc(tot * sizeof(double));
  if (!p->store) return -2;
  double* q = p->store;
  for (int a = 0; a < 3; ++a) {
    int N = dim(c, a);
    oracle_profiles(c, a, q);
    p->be[a] = q; p->ae[a] = q + N; p->ke[a] = q + 2 * N;
    p->bh[a] = q + 3 * N; p->ah[a] = q + 4 * N; p->kh[a] = q + 5 * N;
    q += 6 * N;
  }
  return 0;
}

/* ------------------------------------------------------------ source ----
 * J^{n+1/2} = amplitude * w(u,v) * g((n + 1/2) dt),
 * g(t) = exp(-((t - t0)/tau)^2) sin(w0 (t - t0)), w0 = 2 pi c / lambda0.
 * tau follows from a power-spectrum FWHM of rel_bw * w0:
 * tau = 2 sqrt(2 ln 2) / (rel_bw w0); t0 = t0_over_tau * tau.
 * Everything is expressed in units of dt: w0 dt = 2 pi S dx / lambda0.
 */
int oracle_waveform(const ocfg* c, double* out) {
  double w0dt = 2.0 * M_PI * c->S * c->dx / c->lambda0;
  double tau = 2.0 * sqrt(2.0 * log(2.0)) / (c->rel_bw * w0dt);   /* in steps */
  double t0 = c->t0_over_tau * tau;
  for (int n = 0; n < c->n_steps; ++n) {
    double t = n + 0.5 - t0;
    out[n] = c->amplitude * exp(-(t / tau) * (t / tau)) * sin(w0dt * t);
  }
  return 0;
}

/* Spatial weight of the source on the full grid (component src_comp). */
int oracle_source_weight(const ocfg* c, double* w) {
  memset(w, 0, ncell(c) * sizeof(double));
  if (c->src_kind == 1) {
    w[idx(c, c->src_pos[0], c->src_pos[1], c->src_pos[2])] = 1.0;
  } else if (c->src_kind == 2 || c->src_kind == 3) {
    /* a sheet over the plane's interior cross-section: Gaussian profile
     * (kind 2) or uniform, a normally incident plane wave (kind 3) */
    int a = c->src_axis;
    int ua = a == 0 ? 1 : 0, va = a == 2 ? 1 : 2;
    int P = c->P;
    for (int v = P; v < dim(c, va) - P; ++v)
      for (int u = P; u < dim(c, ua) - P; ++u) {
        double du = (u - c->src_pos[ua]) / c->src_sigma[0];
        double dv = (v - c->src_pos[va]) / c->src_sigma[1];
        int p[3]; p[a] = c->src_pos[a]; p[ua] = u; p[va] = v;
        w[idx(c, p[0], p[1], p[2])] = c->src_kind == 3 ? 1.0 : exp(-0.5 * (du * du + dv * dv));
      }
  }
  return 0;
}

/* --------------------------------------------------------- one step ----
 * state: NF arrays of ncell doubles: Ex Ey Ez Hx Hy Hz psi0..psi11.
 * psi terms (component, derivative axis, differentiated field, sign in curl):
 *   H side: 0 (Hx,y,Ez,+) 1 (Hx,z,Ey,-) 2 (Hy,z,Ex,+) 3 (Hy,x,Ez,-) 4 (Hz,x,Ey,+) 5 (Hz,y,Ex,-)
 *   E side: 6 (Ex,y,Hz,+) 7 (Ex,z,Hy,-) 8 (Ey,z,Hx,+) 9 (Ey,x,Hz,-) 10 (Ez,x,Hy,+) 11 (Ez,y,Hx,-)
 */
typedef struct {
  const ocfg* c;
  oprof pr;
  double* jw;     /* source weight (full grid) */
  double* wave;   /* J waveform per step */
} octx;

static int ctx_init(octx* x, const ocfg* c) {
  x->c = c;
  x->jw = NULL; x->wave = NULL;
  if (prof_alloc(c, &x->pr)) return -2;
  x->jw = (double*)malloc(ncell(c) * sizeof(double));
  x->wave = (double*)malloc((size_t)(c->n_steps > 0 ? c->n_steps : 1) * sizeof(double));
  if (!x->jw || !x->wave) return -2;
  oracle_source_weight(c, x->jw);
  oracle_waveform(c, x->wave);
  return 0;
}

static void ctx_free(octx* x) {
  free(x->pr.store); free(x->jw); free(x->wave);
}

/* H half-step: Ht^{n+1/2} = Ht^{n-1/2} - S * (CPML curl of E^n). */
static void h_update(const octx* x, double* st) {
  const ocfg* c = x->c;
  const oprof* p = &x->pr;
  double *Ex = st, *Ey = st + ncell(c), *Ez = st + 2 * ncell(c);
  double *Hx = st + 3 * ncell(c), *Hy = st + 4 * ncell(c), *Hz = st + 5 * ncell(c);
  double* ps = st + OFF_PSI * ncell(c);
  size_t N = ncell(c);
  double S = c->S;
#pragma omp parallel for schedule(static)
  for (int k = 0; k < c->nz; ++k)
    for (int j = 0; j < c->ny; ++j)
      for (int i = 0; i < c->nx; ++i) {
        size_t q = idx(c, i, j, k);
        double dEz_dy = at(c, Ez, i, j + 1, k) - Ez[q];
        double dEy_dz = at(c, Ey, i, j, k + 1) - Ey[q];
        double dEx_dz = at(c, Ex, i, j, k + 1) - Ex[q];
        double dEz_dx = at(c, Ez, i + 1, j, k) - Ez[q];
        double dEy_dx = at(c, Ey, i + 1, j, k) - Ey[q];
        double dEx_dy = at(c, Ex, i, j + 1, k) - Ex[q];
        double* p0 = &ps[0 * N + q]; double* p1 = &ps[1 * N + q];
        double* p2 = &ps[2 * N + q]; double* p3 = &ps[3 * N + q];
        double* p4 = &ps[4 * N + q]; double* p5 = &ps[5 * N + q];
        *p0 = p->bh[1][j] * *p0 + p->ah[1][j] * dEz_dy;
        *p1 = p->bh[2][k] * *p1 + p->ah[2][k] * dEy_dz;
        *p2 = p->bh[2][k] * *p2 + p->ah[2][k] * dEx_dz;
        *p3 = p->bh[0][i] * *p3 + p->ah[0][i] * dEz_dx;
        *p4 = p->bh[0][i] * *p4 + p->ah[0][i] * dEy_dx;
        *p5 = p->bh[1][j] * *p5 + p->ah[1][j] * dEx_dy;
        double cx = p->kh[1][j] * dEz_dy + *p0 - p->kh[2][k] * dEy_dz - *p1;
        double cy = p->kh[2][k] * dEx_dz + *p2 - p->kh[0][i] * dEz_dx - *p3;
        double cz = p->kh[0][i] * dEy_dx + *p4 - p->kh[1][j] * dEx_dy - *p5;
        Hx[q] -= S * cx;
        Hy[q] -= S * cy;
        Hz[q] -= S * cz;
      }
}

/* E half-step: E^{n+1} = E^n + (S/eps) * (CPML curl of Ht^{n+1/2} - J^{n+1/2}). */
static void e_update(const octx* x, const double* eps, double* st, int n) {
  const ocfg* c = x->c;
  const oprof* p = &x->pr;
  size_t N = ncell(c);
  double *E[3] = {st, st + N, st + 2 * N};
  double *Hx = st + 3 * N, *Hy = st + 4 * N, *Hz = st + 5 * N;
  double* ps = st + OFF_PSI * N;
  double S = c->S;
  double jn = (c->src_kind && n >= 0 && n < c->n_steps) ? x->wave[n] : 0.0;
#pragma omp parallel for schedule(static)
  for (int k = 0; k < c->nz; ++k)
    for (int j = 0; j < c->ny; ++j)
      for (int i = 0; i < c->nx; ++i) {
        size_t q = idx(c, i, j, k);
        double dHz_dy = Hz[q] - at(c, Hz, i, j - 1, k);
        double dHy_dz = Hy[q] - at(c, Hy, i, j, k - 1);
        double dHx_dz = Hx[q] - at(c, Hx, i, j, k - 1);
        double dHz_dx = Hz[q] - at(c, Hz, i - 1, j, k);
        double dHy_dx = Hy[q] - at(c, Hy, i - 1, j, k);
        double dHx_dy = Hx[q] - at(c, Hx, i, j - 1, k);
        double* p6 = &ps[6 * N + q]; double* p7 = &ps[7 * N + q];
        double* p8 = &ps[8 * N + q]; double* p9 = &ps[9 * N + q];
        double* p10 = &ps[10 * N + q]; double* p11 = &ps[11 * N + q];
        *p6 = p->be[1][j] * *p6 + p->ae[1][j] * dHz_dy;
        *p7 = p->be[2][k] * *p7 + p->ae[2][k] * dHy_dz;
        *p8 = p->be[2][k] * *p8 + p->ae[2][k] * dHx_dz;
        *p9 = p->be[0][i] * *p9 + p->ae[0][i] * dHz_dx;
        *p10 = p->be[0][i] * *p10 + p->ae[0][i] * dHy_dx;
        *p11 = p->be[1][j] * *p11 + p->ae[1][j] * dHx_dy;
        double curl[3];
        curl[0] = p->ke[1][j] * dHz_dy + *p6 - p->ke[2][k] * dHy_dz - *p7;
        curl[1] = p->ke[2][k] * dHx_dz + *p8 - p->ke[0][i] * dHz_dx - *p9;
        curl[2] = p->ke[0][i] * dHy_dx + *p10 - p->ke[1][j] * dHx_dy - *p11;
        if (c->src_kind) curl[c->src_comp] -= x->jw[q] * jn;
        double cb = S / eps[q];
        for (int e = 0; e < 3; ++e) E[e][q] += cb * curl[e];
      }
}

/* Detector plane iteration: calls back with the cell index of every (u,v). */
static void det_cell(const ocfg* c, int u, int v, int* i, int* j, int* k) {
  int p[3]; int a = c->det_axis;
  int ua = a == 0 ? 1 : 0, va = a == 2 ? 1 : 2;
  p[a] = c->det_index; p[ua] = u; p[va] = v;
  *i = p[0]; *j = p[1]; *k = p[2];
}

/* l_n = sum over the plane of |E|^2 (kind 1) or of (E x Ht) . n (kind 2),
 * fields co-indexed at each cell. */
static double objective(const ocfg* c, const double* st) {
  size_t N = ncell(c);
  const double *E = st, *H = st + 3 * N;
  int a = c->det_axis, b = (a + 1) % 3, d = (a + 2) % 3;
  double L = 0.0;
  for (int v = c->det_lo[1]; v < c->det_hi[1]; ++v)
    for (int u = c->det_lo[0]; u < c->det_hi[0]; ++u) {
      int i, j, k; det_cell(c, u, v, &i, &j, &k);
      size_t q = idx(c, i, j, k);
      if (c->det_kind == 1)
        L += E[q] * E[q] + E[N + q] * E[N + q] + E[2 * N + q] * E[2 * N + q];
      else
        L += E[b * N + q] * H[d * N + q] - E[d * N + q] * H[b * N + q];
    }
  return L;
}

/* lambda += seed * dl/d(E^{n+1}, Ht^{n+1/2}) given the primal plane fields. */
static void objective_seed(const ocfg* c, const double* st, double seed, double* lam) {
  size_t N = ncell(c);
  const double *E = st, *H = st + 3 * N;
  double *lE = lam, *lH = lam + 3 * N;
  int a = c->det_axis, b = (a + 1) % 3, d = (a + 2) % 3;
  for (int v = c->det_lo[1]; v < c->det_hi[1]; ++v)
    for (int u = c->det_lo[0]; u < c->det_hi[0]; ++u) {
      int i, j, k; det_cell(c, u, v, &i, &j, &k);
      size_t q = idx(c, i, j, k);
      if (c->det_kind == 1) {
        for (int e = 0; e < 3; ++e) lE[e * N + q] += seed * 2.0 * E[e * N + q];
      } else {
        lE[b * N + q] += seed * H[d * N + q];
        lE[d * N + q] -= seed * H[b * N + q];
        lH[d * N + q] += seed * E[b * N + q];
        lH[b * N + q] -= seed * E[d * N + q];
      }
    }
}

/* Public single step (state in place). Returns l_n via *obj if non-NULL. */
int oracle_step(const ocfg* c, const double* eps, double* st, int n, double* obj) {
  octx x;
  if (ctx_init(&x, c)) { ctx_free(&x); return -2; }
  h_update(&x, st);
  e_update(&x, eps, st, n);
  if (obj) *obj = c->det_kind ? objective(c, st) : 0.0;
  ctx_free(&x);
  return 0;
}

/* Run steps n0 .. n0+count-1 from the given state; obj[count] per-step l_n. */
int oracle_run(const ocfg* c, const double* eps, double* st, int n0, int count, double* obj) {
  octx x;
  if (ctx_init(&x, c)) { ctx_free(&x); return -2; }
  for (int s = 0; s < count; ++s) {
    h_update(&x, st);
    e_update(&x, eps, st, n0 + s);
    if (obj) obj[s] = c->det_kind ? objective(c, st) : 0.0;
  }
  ctx_free(&x);
  return 0;
}

/* ------------------------------------------------- adjoint of one step ----
 * Transpose of the step above, applied to the adjoint state lam (same NF
 * layout).  The E half-step is transposed first, then the H half-step.
 * Per psi term t with sign s:  mu = lam_psi + (coefficient) * lam_field,
 * lam_delta = (coefficient) * kinv * lam_field + a * mu,  lam_psi <- b * mu,
 * and the difference operator's transpose moves lam_delta onto the
 * differentiated field: D'^T g (c) = g(c) - g(c+1) for backward differences,
 * D^T g (c) = g(c-1) - g(c) for forward differences (zero outside).
 * If gcb != NULL and dE != NULL, accumulates sum_e lam_E[e] * dE[e] / cb,
 * i.e. dL/d(cb) with dE = E^{n+1} - E^n supplied by the caller.
 */
static void adj_e_transpose(const octx* x, const double* eps, double* lam, double* tmp) {
  const ocfg* c = x->c;
  const oprof* p = &x->pr;
  size_t N = ncell(c);
  double *lE = lam, *lH = lam + 3 * N, *lp = lam + OFF_PSI * N;
  double S = c->S;
  /* tmp: 6 arrays lam_delta for terms 6..11 */
#pragma omp parallel for schedule(static)
  for (int k = 0; k < c->nz; ++k)
    for (int j = 0; j < c->ny; ++j)
      for (int i = 0; i < c->nx; ++i) {
        size_t q = idx(c, i, j, k);
        double cb = S / eps[q];
        /* term: (psi index, E comp, axis, sign) */
        const int tE[6] = {0, 0, 1, 1, 2, 2};
        const int tA[6] = {1, 2, 2, 0, 0, 1};
        const double tS[6] = {+1, -1, +1, -1, +1, -1};
        for (int t = 0; t < 6; ++t) {
          int ax = tA[t];
          int pos = ax == 0 ? i : (ax == 1 ? j : k);
          double le = lE[tE[t] * N + q];
          double mu = lp[(6 + t) * N + q] + tS[t] * cb * le;
          tmp[t * N + q] = tS[t] * cb * p->ke[ax][pos] * le + p->ae[ax][pos] * mu;
          lp[(6 + t) * N + q] = p->be[ax][pos] * mu;
        }
      }
  /* lam_H += D'^T lam_delta: term 6 (d/dy Hz), 7 (d/dz Hy), 8 (d/dz Hx),
   * 9 (d/dx Hz), 10 (d/dx Hy), 11 (d/dy Hx). */
#pragma omp parallel for schedule(static)
  for (int k = 0; k < c->nz; ++k)
    for (int j = 0; j < c->ny; ++j)
      for (int i = 0; i < c->nx; ++i) {
        size_t q = idx(c, i, j, k);
        double* d6 = tmp; double* d7 = tmp + N; double* d8 = tmp + 2 * N;
        double* d9 = tmp + 3 * N; double* d10 = tmp + 4 * N; double* d11 = tmp + 5 * N;
        lH[0 * N + q] += (d8[q] - at(c, d8, i, j, k + 1)) + (d11[q] - at(c, d11, i, j + 1, k));
        lH[1 * N + q] += (d7[q] - at(c, d7, i, j, k + 1)) + (d10[q] - at(c, d10, i + 1, j, k));
        lH[2 * N + q] += (d6[q] - at(c, d6, i, j + 1, k)) + (d9[q] - at(c, d9, i + 1, j, k));
      }
}

static void adj_h_transpose(const octx* x, double* lam, double* tmp) {
  const ocfg* c = x->c;
  const oprof* p = &x->pr;
  size_t N = ncell(c);
  double *lE = lam, *lH = lam + 3 * N, *lp = lam + OFF_PSI * N;
  double S = c->S;
#pragma omp parallel for schedule(static)
  for (int k = 0; k < c->nz; ++k)
    for (int j = 0; j < c->ny; ++j)
      for (int i = 0; i < c->nx; ++i) {
        size_t q = idx(c, i, j, k);
        const int tH[6] = {0, 0, 1, 1, 2, 2};
        const int tA[6] = {1, 2, 2, 0, 0, 1};
        const double tS[6] = {+1, -1, +1, -1, +1, -1};
        for (int t = 0; t < 6; ++t) {
          int ax = tA[t];
          int pos = ax == 0 ? i : (ax == 1 ? j : k);
          double lh = lH[tH[t] * N + q];
          double mu = lp[t * N + q] - S * tS[t] * lh;
          tmp[t * N + q] = -S * tS[t] * p->kh[ax][pos] * lh + p->ah[ax][pos] * mu;
          lp[t * N + q] = p->bh[ax][pos] * mu;
        }
      }
  /* lam_E += D^T lam_delta: term 0 (d/dy Ez), 1 (d/dz Ey), 2 (d/dz Ex),
   * 3 (d/dx Ez), 4 (d/dx Ey), 5 (d/dy Ex). */
#pragma omp parallel for schedule(static)
  for (int k = 0; k < c->nz; ++k)
    for (int j = 0; j < c->ny; ++j)
      for (int i = 0; i < c->nx; ++i) {
        size_t q = idx(c, i, j, k);
        double* d0 = tmp; double* d1 = tmp + N; double* d2 = tmp + 2 * N;
        double* d3 = tmp + 3 * N; double* d4 = tmp + 4 * N; double* d5 = tmp + 5 * N;
        lE[0 * N + q] += (at(c, d2, i, j, k - 1) - d2[q]) + (at(c, d5, i, j - 1, k) - d5[q]);
        lE[1 * N + q] += (at(c, d1, i, j, k - 1) - d1[q]) + (at(c, d4, i - 1, j, k) - d4[q]);
        lE[2 * N + q] += (at(c, d0, i, j - 1, k) - d0[q]) + (at(c, d3, i - 1, j, k) - d3[q]);
      }
}

/* Public: lam <- F^T lam for one source-free step (dot-product tests). */
int oracle_step_adjoint(const ocfg* c, const double* eps, double* lam) {
  octx x;
  if (ctx_init(&x, c)) { ctx_free(&x); return -2; }
  double* tmp = (double*)malloc(6 * ncell(c) * sizeof(double));
  if (!tmp) { ctx_free(&x); return -2; }
  adj_e_transpose(&x, eps, lam, tmp);
  adj_h_transpose(&x, lam, tmp);
  free(tmp);
  ctx_free(&x);
  return 0;
}

/* ------------------------------------------- stored-history gradient ----
 * Forward N steps from the zero state, keeping E inside the design box at
 * every step and the detector-plane fields; then the adjoint from n = N-1
 * down to 0.  dL/d(eps) = -sum_n sum_e lam_E^{n+1}[e] (E^{n+1}-E^n)[e] / eps,
 * because E^{n+1} = E^n + (S/eps) X and d(S/eps)/d(eps) = -(S/eps)/eps.
 * grad: design box [dz][dy][dx], multiplied by seed.  obj: L.
 */
/* The second detector as a configuration of its own (same grid, det_* of
 * the second detector), so the plane helpers above serve both. */
static ocfg second_detector(const ocfg* c) {
  ocfg d = *c;
  d.det_kind = c->det2_kind;
  d.det_axis = c->det2_axis;
  d.det_index = c->det2_index;
  d.det_lo[0] = c->det2_lo[0]; d.det_lo[1] = c->det2_lo[1];
  d.det_hi[0] = c->det2_hi[0]; d.det_hi[1] = c->det2_hi[1];
  return d;
}

/* Stored-history gradient of seed * L + seed2 * M (M from the second
 * detector when det2_kind != 0).  obj2 (optional): {L, M}. */
int oracle_gradient2(const ocfg* c, const double* eps, double seed, double seed2, double* grad,
                     double* obj2, double* final_state) {
  size_t N = ncell(c);
  int dX = c->dhi[0] - c->dlo[0], dY = c->dhi[1] - c->dlo[1], dZ = c->dhi[2] - c->dlo[2];
  size_t nd = (size_t)dX * dY * dZ;
  int T = c->n_steps;
  const ocfg c2 = second_detector(c);
  const int nd2 = c->det2_kind ? 2 : 1;
  const ocfg* dc[2] = {c, &c2};
  int nu[2], nv[2];
  size_t np[2];
  for (int t = 0; t < 2; ++t) {
    nu[t] = dc[t]->det_hi[0] - dc[t]->det_lo[0];
    nv[t] = dc[t]->det_hi[1] - dc[t]->det_lo[1];
    np[t] = t < nd2 ? (size_t)nu[t] * nv[t] : 0;
  }
  octx x;
  if (ctx_init(&x, c)) { ctx_free(&x); return -2; }
  double* st = (double*)calloc(NF * N, sizeof(double));
  double* lam = (double*)calloc(NF * N, sizeof(double));
  double* tmp = (double*)malloc(6 * N * sizeof(double));
  double* hist = (double*)malloc((size_t)(T + 1) * 3 * nd * sizeof(double));
  double* dets = (double*)malloc((size_t)T * 6 * (np[0] + np[1]) * sizeof(double));
  double* plane = (double*)calloc(NF * N, sizeof(double));   /* scratch for seeds */
  if (!st || !lam || !tmp || !hist || !dets || !plane) {
    free(st); free(lam); free(tmp); free(hist); free(dets); free(plane); ctx_free(&x);
    return -2;
  }
#define SAVE_DESIGN(slot)                                                        \
  for (int e = 0; e < 3; ++e)                                                    \
    for (int kk = 0; kk < dZ; ++kk)                                              \
      for (int jj = 0; jj < dY; ++jj)                                            \
        for (int ii = 0; ii < dX; ++ii)                                          \
          hist[((size_t)(slot) * 3 + e) * nd + ((size_t)kk * dY + jj) * dX + ii] = \
              st[e * N + idx(c, c->dlo[0] + ii, c->dlo[1] + jj, c->dlo[2] + kk)];
  /* detector t's plane fields of step n live at dets + n*6*(np0+np1) + t*6*np0 */
#define DET_AT(n, t, f, v, u) \
  dets[(size_t)(n) * 6 * (np[0] + np[1]) + (size_t)(t) * 6 * np[0] + (size_t)(f) * np[t] + \
       (size_t)(v) * nu[t] + (u)]
  double Ls[2] = {0.0, 0.0};
  SAVE_DESIGN(0);
  for (int n = 0; n < T; ++n) {
    h_update(&x, st);
    e_update(&x, eps, st, n);
    for (int t = 0; t < nd2; ++t) {
      Ls[t] += objective(dc[t], st);
      for (int f = 0; f < 6; ++f)
        for (int v = 0; v < nv[t]; ++v)
          for (int u = 0; u < nu[t]; ++u) {
            int i, j, k;
            det_cell(dc[t], dc[t]->det_lo[0] + u, dc[t]->det_lo[1] + v, &i, &j, &k);
            DET_AT(n, t, f, v, u) = st[f * N + idx(c, i, j, k)];
          }
    }
    SAVE_DESIGN(n + 1);
  }
  if (final_state) memcpy(final_state, st, NF * N * sizeof(double));
  for (size_t q = 0; q < nd; ++q) grad[q] = 0.0;
  const double seeds[2] = {seed, seed2};
  for (int n = T - 1; n >= 0; --n) {
    /* seed from the stored plane fields (E^{n+1}, Ht^{n+1/2}) of each detector */
    for (int t = 0; t < nd2; ++t) {
      for (int f = 0; f < 6; ++f)
        for (int v = 0; v < nv[t]; ++v)
          for (int u = 0; u < nu[t]; ++u) {
            int i, j, k;
            det_cell(dc[t], dc[t]->det_lo[0] + u, dc[t]->det_lo[1] + v, &i, &j, &k);
            plane[f * N + idx(c, i, j, k)] = DET_AT(n, t, f, v, u);
          }
      objective_seed(dc[t], plane, seeds[t], lam);
    }
    /* gradient with lam_E^{n+1} (seeded, before this step's transposes) */
    for (int kk = 0; kk < dZ; ++kk)
      for (int jj = 0; jj < dY; ++jj)
        for (int ii = 0; ii < dX; ++ii) {
          size_t qd = ((size_t)kk * dY + jj) * dX + ii;
          size_t q = idx(c, c->dlo[0] + ii, c->dlo[1] + jj, c->dlo[2] + kk);
          double s = 0.0;
          for (int e = 0; e < 3; ++e) {
            double dE = hist[((size_t)(n + 1) * 3 + e) * nd + qd] - hist[((size_t)n * 3 + e) * nd + qd];
            s += lam[e * N + q] * dE;
          }
          grad[qd] += -s / eps[q];
        }
    adj_e_transpose(&x, eps, lam, tmp);
    adj_h_transpose(&x, lam, tmp);
  }
#undef SAVE_DESIGN
#undef DET_AT
  if (obj2) { obj2[0] = Ls[0]; obj2[1] = Ls[1]; }
  free(st); free(lam); free(tmp); free(hist); free(dets); free(plane);
  ctx_free(&x);
  return 0;
}

/* The single-objective gradient: seed * dL/d(eps) (second detector ignored). */
int oracle_gradient(const ocfg* c, const double* eps, double seed, double* grad, double* obj,
                    double* final_state) {
  ocfg one = *c;
  one.det2_kind = 0;
  double o2[2];
  int rc = oracle_gradient2(&one, eps, seed, 0.0, grad, o2, final_state);
  if (obj) *obj = o2[0];
  return rc;
}

/* ----------------------------------------------------- quantisers ----
 * Round-to-nearest-even of a double onto a binary floating-point format with
 * `mbits` stored mantissa bits, smallest normal exponent `emin` (subnormals
 * below it share the spacing 2^(emin-mbits)) and largest finite value `fmax`;
 * results above fmax saturate to fmax (satfinite).  Formats (IEEE / OCP):
 *   1 bfloat16: 7 mantissa bits, emin -126, max (2 - 2^-7) 2^127
 *   2 float16 : 10 mantissa bits, emin -14, max 65504
 *   3 float8 e4m3fn: 3 mantissa bits, emin -6, max 448
 *   0 float32 : 23 mantissa bits, emin -126 (the FP32 tape)
 * The 8-bit formats the paper compares in Sec. 4 (Fig. 3); for an exponent
 * field of E bits with bias B the smallest normal exponent is 1 - B.  "fnuz"
 * formats have no infinities and one NaN code (0x80), so every other code,
 * the all-ones exponent included, is finite; the IEEE-like formats reserve
 * the all-ones exponent for infinities and NaNs:
 *   4 float8 e4m3b11fnuz: 3 mantissa bits, bias 11, emin -10, max 1.875 * 2^4 = 30
 *   5 float8 e5m2fnuz   : 2 mantissa bits, bias 16, emin -15, max 1.75 * 2^15 = 57344
 *   6 float8 e4m3fnuz   : 3 mantissa bits, bias 8,  emin -7,  max 1.875 * 2^7 = 240
 *   7 float8 e4m3 (IEEE): 3 mantissa bits, bias 7,  emin -6,  max 1.875 * 2^7 = 240
 *   8 float8 e3m4 (IEEE): 4 mantissa bits, bias 3,  emin -2,  max 1.9375 * 2^3 = 15.5
 * Saturation of out-of-range values is this implementation's reading (the
 * paper does not say how values beyond the range are converted).
 */
static double quant_generic(double x, int mbits, int emin, double fmax) {
  if (x == 0.0 || isnan(x)) return x;
  double ax = fabs(x);
  int e;
  frexp(ax, &e);                 /* ax = f * 2^e, f in [0.5, 1): exponent = e - 1 */
  int ex = e - 1;
  if (ex < emin) ex = emin;
  double ulp = ldexp(1.0, ex - mbits);
  double q = nearbyint(ax / ulp) * ulp;   /* default rounding mode: ties to even */
  if (q > fmax) q = fmax;
  return x < 0 ? -q : q;
}

double oracle_format_max(int fmt) {
  switch (fmt) {
    case 0: return ldexp(2.0 - ldexp(1.0, -23), 127);
    case 1: return ldexp(2.0 - ldexp(1.0, -7), 127);
    case 2: return 65504.0;
    case 3: return 448.0;
    case 4: return 30.0;
    case 5: return 57344.0;
    case 6: return 240.0;
    case 7: return 240.0;
    case 8: return 15.5;
  }
  return 0.0;
}

double oracle_quantize(int fmt, double x) {
  switch (fmt) {
    case 0: return quant_generic(x, 23, -126, oracle_format_max(0));
    case 1: return quant_generic(x, 7, -126, oracle_format_max(1));
    case 2: return quant_generic(x, 10, -14, 65504.0);
    case 3: return quant_generic(x, 3, -6, 448.0);
    case 4: return quant_generic(x, 3, -10, 30.0);
    case 5: return quant_generic(x, 2, -15, 57344.0);
    case 6: return quant_generic(x, 3, -7, 240.0);
    case 7: return quant_generic(x, 3, -6, 240.0);
    case 8: return quant_generic(x, 4, -2, 15.5);
  }
  return x;
}

int oracle_quantize_array(int fmt, const double* in, double* out, long n) {
  for (long i = 0; i < n; ++i) out[i] = oracle_quantize(fmt, in[i]);
  return 0;
}

/* ------------------------------------------ block-transform codec ----
 * Beyond the paper (its Sec. 4 names JPEG-like compression of the tape as
 * future work): a face component [v][u] is cut into 8 x 8 blocks, cells past
 * the face edge repeating the last row / column; each block is expanded in
 * the orthonormal 2D DCT-II basis
 *     B_uv(x, y) = c_u c_v cos((2x+1) u pi/16) cos((2y+1) v pi/16),
 *     c_0 = sqrt(1/8), c_u = sqrt(2/8) otherwise,
 * and only the first K coefficients in diagonal order (u + v ascending, then
 * v ascending) are kept, each as an int8 code round(C / s) with the block
 * scale s = max(max|C| / 127, 2^-126) (1 for an all-zero block).
 * This is a quantised code decided in floating point, so it is computed in
 * the precision the CUDA path uses: float32, the basis rounded to float from
 * the double product, every sum an fmaf chain in a fixed order (cells row by
 * row for a coefficient; kept coefficients in order for a value), then one
 * float multiply by s.  (The cross-check against an FP64 DCT is a test.)
 */
static void bdct_uv(int i, int* u, int* v) {
  int n = 0;
  for (int d = 0; d <= 14; ++d)
    for (int vv = 0; vv <= d && vv <= 7; ++vv) {
      int uu = d - vv;
      if (uu > 7) continue;
      if (n++ == i) { *u = uu; *v = vv; return; }
    }
  *u = 0; *v = 0;
}

/* beta[i*64 + y*8 + x] = B_{u_i v_i}(x, y) as float. */
void oracle_bdct_basis(float* beta) {
  for (int i = 0; i < 64; ++i) {
    int u, v; bdct_uv(i, &u, &v);
    for (int y = 0; y < 8; ++y)
      for (int x = 0; x < 8; ++x) {
        double cu = u == 0 ? sqrt(1.0 / 8.0) : 0.5, cv = v == 0 ? sqrt(1.0 / 8.0) : 0.5;
        double du = cu * cos((2 * x + 1) * u * 3.14159265358979323846 / 16.0);
        double dv = cv * cos((2 * y + 1) * v * 3.14159265358979323846 / 16.0);
        beta[i * 64 + y * 8 + x] = (float)(du * dv);
      }
  }
}

/* in [nv][nu] -> codes [nblocks][K] and scales [nblocks], blocks row-major. */
int oracle_bdct_encode(const float* in, int nu, int nv, int K, signed char* codes, float* scales) {
  if (nu < 1 || nv < 1 || K < 1 || K > 64) return -1;
  float beta[64 * 64];
  oracle_bdct_basis(beta);
  int nbu = (nu + 7) / 8, nbv = (nv + 7) / 8;
  for (int bv = 0; bv < nbv; ++bv)
    for (int bu = 0; bu < nbu; ++bu) {
      float X[64], C[64];
      for (int y = 0; y < 8; ++y)
        for (int x = 0; x < 8; ++x) {
          int vv = bv * 8 + y < nv ? bv * 8 + y : nv - 1;
          int uu = bu * 8 + x < nu ? bu * 8 + x : nu - 1;
          X[y * 8 + x] = in[(size_t)vv * nu + uu];
        }
      float amax = 0.0f;
      for (int i = 0; i < K; ++i) {
        float c = 0.0f;
        for (int t = 0; t < 64; ++t) c = fmaf(X[t], beta[i * 64 + t], c);
        C[i] = c;
        if (fabsf(c) > amax) amax = fabsf(c);
      }
      float s = 1.0f;
      if (amax > 0.0f) {
        s = amax / 127.0f;
        if (s < 1.17549435e-38f) s = 1.17549435e-38f;
      }
      size_t b = (size_t)bv * nbu + bu;
      for (int i = 0; i < K; ++i) {
        float q = rintf(C[i] / s);
        if (q > 127.0f) q = 127.0f;
        if (q < -127.0f) q = -127.0f;
        codes[b * K + i] = (signed char)(int)q;
      }
      scales[b] = s;
    }
  return 0;
}

int oracle_bdct_decode(const signed char* codes, const float* scales, int nu, int nv, int K,
                       float* out) {
  if (nu < 1 || nv < 1 || K < 1 || K > 64) return -1;
  float beta[64 * 64];
  oracle_bdct_basis(beta);
  int nbu = (nu + 7) / 8;
  for (int vv = 0; vv < nv; ++vv)
    for (int uu = 0; uu < nu; ++uu) {
      size_t b = (size_t)(vv / 8) * nbu + uu / 8;
      int t = (vv % 8) * 8 + uu % 8;
      float acc = 0.0f;
      for (int i = 0; i < K; ++i) acc = fmaf((float)codes[b * K + i], beta[i * 64 + t], acc);
      out[(size_t)vv * nu + uu] = acc * scales[b];
    }
  return 0;
}

/* Apply the codec to one face sample in place ([comp][v][u], float32 values
 * as the CUDA path records them). */
static int bdct_face(double* v, int nu, int nv, int K) {
  size_t n = (size_t)nu * nv;
  int nb = ((nu + 7) / 8) * ((nv + 7) / 8);
  float* x = (float*)malloc(n * sizeof(float));
  float* y = (float*)malloc(n * sizeof(float));
  signed char* codes = (signed char*)malloc((size_t)nb * K);
  float* sc = (float*)malloc((size_t)nb * sizeof(float));
  if (!x || !y || !codes || !sc) { free(x); free(y); free(codes); free(sc); return -2; }
  for (int t = 0; t < 2; ++t) {
    for (size_t i = 0; i < n; ++i) x[i] = (float)v[t * n + i];
    oracle_bdct_encode(x, nu, nv, K, codes, sc);
    oracle_bdct_decode(codes, sc, nu, nv, K, y);
    for (size_t i = 0; i < n; ++i) v[t * n + i] = y[i];
  }
  free(x); free(y); free(codes); free(sc);
  return 0;
}

/* ------------------------------------------------- interpolation ----
 * Value at time q of a series known at increasing knots t[0..nk-1].
 * kind 0: linear between the bracketing knots (Sec. 2).
 * kind 1: cubic Hermite whose knot slopes are those of the quadratic through
 *   the knot and its two neighbours (one-sided at the first and last knot);
 *   on a uniform grid this is Catmull-Rom.  Exact for quadratics.
 * q outside [t0, t_{nk-1}] clamps to the end value.
 */
static double slope_at(const double* t, const double* p, int nk, int j) {
  if (nk < 2) return 0.0;
  if (nk == 2) return (p[1] - p[0]) / (t[1] - t[0]);
  if (j == 0) {
    double h0 = t[1] - t[0], h1 = t[2] - t[1];
    return -(2 * h0 + h1) / (h0 * (h0 + h1)) * p[0] + (h0 + h1) / (h0 * h1) * p[1]
           - h0 / (h1 * (h0 + h1)) * p[2];
  }
  if (j == nk - 1) {
    double ha = t[j - 1] - t[j - 2], hb = t[j] - t[j - 1];
    return hb / (ha * (ha + hb)) * p[j - 2] - (ha + hb) / (ha * hb) * p[j - 1]
           + (2 * hb + ha) / (hb * (ha + hb)) * p[j];
  }
  double hl = t[j] - t[j - 1], hr = t[j + 1] - t[j];
  return -hr / (hl * (hl + hr)) * p[j - 1] + (hr - hl) / (hl * hr) * p[j]
         + hl / (hr * (hl + hr)) * p[j + 1];
}

static double interp_eval(int kind, const double* t, const double* p, int nk, double q) {
  if (nk <= 0) return 0.0;
  if (q <= t[0]) return p[0];
  if (q >= t[nk - 1]) return p[nk - 1];
  int a = 0;
  while (!(t[a] <= q && q <= t[a + 1])) ++a;
  if (q == t[a]) return p[a];
  if (q == t[a + 1]) return p[a + 1];
  double h = t[a + 1] - t[a];
  double s = (q - t[a]) / h;
  if (kind == 0) return (1.0 - s) * p[a] + s * p[a + 1];
  double ma = slope_at(t, p, nk, a), mb = slope_at(t, p, nk, a + 1);
  double h00 = 2 * s * s * s - 3 * s * s + 1, h10 = s * s * s - 2 * s * s + s;
  double h01 = -2 * s * s * s + 3 * s * s, h11 = s * s * s - s * s;
  return h00 * p[a] + h10 * h * ma + h01 * p[a + 1] + h11 * h * mb;
}

int oracle_interp_series(int kind, int nk, const double* t, const double* p, int nq,
                         const double* q, double* out) {
  for (int i = 0; i < nq; ++i) out[i] = interp_eval(kind, t, p, nk, q[i]);
  return 0;
}

/* -------------------------------------------- interface-slice tape ----
 * The layers the interior inverse needs from outside the interior
 * I = [P, N-P)^3 (Sec. 2: fields on the interface slices between the
 * simulation volume and the PML):
 *   low faces  (x-, y-, z-) at index P-1: the two tangential Ht components at
 *              half-step n+1/2 (read by the inverse E update at index P);
 *   high faces (x+, y+, z+) at index N-P: the two tangential E components at
 *              step n (read by the inverse H update at index N-P-1).
 * Each face spans the interior cross-section.  Face f = 2*axis + (high?1:0);
 * tangential components in increasing axis order; values [comp][v][u].
 */
static void face_dims(const ocfg* c, int f, int* ua, int* va, int* nu, int* nv) {
  int a = f / 2;
  *ua = a == 0 ? 1 : 0; *va = a == 2 ? 1 : 2;
  *nu = dim(c, *ua) - 2 * c->P; *nv = dim(c, *va) - 2 * c->P;
}

static size_t face_values(const ocfg* c, int f) {
  int ua, va, nu, nv; face_dims(c, f, &ua, &va, &nu, &nv);
  return 2 * (size_t)nu * nv;
}

size_t oracle_sample_values(const ocfg* c) {
  size_t s = 0;
  for (int f = 0; f < 6; ++f) s += face_values(c, f);
  return s;
}

/* Copy (dir=0: state -> buf) or (dir=1: buf -> state) the layer of face f. */
static void face_io(const ocfg* c, int f, double* st, double* buf, int dir) {
  int a = f / 2, high = f % 2;
  int ua, va, nu, nv; face_dims(c, f, &ua, &va, &nu, &nv);
  size_t N = ncell(c);
  int layer = high ? dim(c, a) - c->P : c->P - 1;
  int base = high ? OFF_E : OFF_H;
  int comps[2] = {ua, va};
  for (int t = 0; t < 2; ++t)
    for (int v = 0; v < nv; ++v)
      for (int u = 0; u < nu; ++u) {
        int p[3]; p[a] = layer; p[ua] = c->P + u; p[va] = c->P + v;
        double* fld = st + (size_t)(base + comps[t]) * N + idx(c, p[0], p[1], p[2]);
        double* b = buf + ((size_t)t * nv + v) * nu + u;
        if (dir == 0) *b = *fld; else *fld = *b;
      }
}

/* Quantise one face sample in place: optional per-face absmax scale. */
static void encode_face(int fmt, int scaled, double* v, size_t n, double* scale_out) {
  double scale = 1.0;
  if (scaled) {
    double amax = 0.0;
    for (size_t i = 0; i < n; ++i) amax = fmax(amax, fabs(v[i]));
    /* at least the smallest normal FP32 number (2^-126), as stored scales are FP32 */
    scale = amax > 0.0 ? fmax(amax / oracle_format_max(fmt), ldexp(1.0, -126)) : 1.0;
  }
  for (size_t i = 0; i < n; ++i) v[i] = oracle_quantize(fmt, v[i] / scale) * scale;
  if (scale_out) *scale_out = scale;
}

/* Public: the face encoder on one array (for its tests). */
void oracle_encode_face(int fmt, int scaled, double* v, size_t n, double* scale_out) {
  encode_face(fmt, scaled, v, n, scale_out);
}

/* Inverse interior updates: E^n from (E^{n+1}, Ht^{n+1/2}), then Ht^{n-1/2}
 * from (Ht^{n+1/2}, E^n).  Only cells of I are written; the interior has
 * kappa = 1 and no psi, so the curls are the plain lossless ones.
 * dE (optional, 3*ncell) receives E^{n+1} - E^n on I. */
static void inverse_e(const octx* x, const double* eps, double* st, int n, double* dE) {
  const ocfg* c = x->c;
  size_t N = ncell(c);
  double *E[3] = {st, st + N, st + 2 * N};
  double *Hx = st + 3 * N, *Hy = st + 4 * N, *Hz = st + 5 * N;
  int P = c->P;
  double jn = (c->src_kind && n >= 0 && n < c->n_steps) ? x->wave[n] : 0.0;
#pragma omp parallel for schedule(static)
  for (int k = P; k < c->nz - P; ++k)
    for (int j = P; j < c->ny - P; ++j)
      for (int i = P; i < c->nx - P; ++i) {
        size_t q = idx(c, i, j, k);
        double curl[3];
        curl[0] = (Hz[q] - at(c, Hz, i, j - 1, k)) - (Hy[q] - at(c, Hy, i, j, k - 1));
        curl[1] = (Hx[q] - at(c, Hx, i, j, k - 1)) - (Hz[q] - at(c, Hz, i - 1, j, k));
        curl[2] = (Hy[q] - at(c, Hy, i - 1, j, k)) - (Hx[q] - at(c, Hx, i, j - 1, k));
        if (c->src_kind) curl[c->src_comp] -= x->jw[q] * jn;
        double cb = c->S / eps[q];
        for (int e = 0; e < 3; ++e) {
          double d = cb * curl[e];
          E[e][q] -= d;
          if (dE) dE[e * N + q] = d;
        }
      }
}

static void inverse_h(const octx* x, double* st) {
  const ocfg* c = x->c;
  size_t N = ncell(c);
  double *Ex = st, *Ey = st + N, *Ez = st + 2 * N;
  double *Hx = st + 3 * N, *Hy = st + 4 * N, *Hz = st + 5 * N;
  int P = c->P;
  double S = c->S;
#pragma omp parallel for schedule(static)
  for (int k = P; k < c->nz - P; ++k)
    for (int j = P; j < c->ny - P; ++j)
      for (int i = P; i < c->nx - P; ++i) {
        size_t q = idx(c, i, j, k);
        Hx[q] += S * ((at(c, Ez, i, j + 1, k) - Ez[q]) - (at(c, Ey, i, j, k + 1) - Ey[q]));
        Hy[q] += S * ((at(c, Ex, i, j, k + 1) - Ex[q]) - (at(c, Ez, i + 1, j, k) - Ez[q]));
        Hz[q] += S * ((at(c, Ey, i + 1, j, k) - Ey[q]) - (at(c, Ex, i, j + 1, k) - Ex[q]));
      }
}

/* Public: invert step n on the interior in place (P = 0: the whole grid). */
int oracle_unstep(const ocfg* c, const double* eps, double* st, int n) {
  octx x;
  if (ctx_init(&x, c)) { ctx_free(&x); return -2; }
  inverse_e(&x, eps, st, n, NULL);
  inverse_h(&x, st);
  ctx_free(&x);
  return 0;
}

/* grad += -sum_e lam_E[e] * dE[e] / eps on the design box [dz][dy][dx]
 * (dE = E^{n+1} - E^n = cb * (curl Ht - J): the adjoint's share of step n). */
static void grad_accumulate(const ocfg* c, const double* eps, const double* lam,
                            const double* dE, double* grad) {
  size_t N = ncell(c);
  int dX = c->dhi[0] - c->dlo[0], dY = c->dhi[1] - c->dlo[1], dZ = c->dhi[2] - c->dlo[2];
  for (int kk = 0; kk < dZ; ++kk)
    for (int jj = 0; jj < dY; ++jj)
      for (int ii = 0; ii < dX; ++ii) {
        size_t q = idx(c, c->dlo[0] + ii, c->dlo[1] + jj, c->dlo[2] + kk);
        double s = 0.0;
        for (int e = 0; e < 3; ++e) s += lam[e * N + q] * dE[e * N + q];
        grad[((size_t)kk * dY + jj) * dX + ii] += -s / eps[q];
      }
}

/* ------------------------------------------------ the method, FP64 ----
 * Forward N steps recording the interface slices at the sample steps
 * s_j = r + j k (r = (N-1) mod k, so the last step is always a sample),
 * each face quantised to `fmt` (optionally with a per-face, per-sample absmax
 * scale).  Then the time-reversed simulation with the adjoint:
 *   for n = N-1 .. 0:
 *     restore Ht^{n+1/2} on the low layers (interpolated over the samples and
 *       the known zero state Ht^{-1/2} at time -1);
 *     seed lam with dl_n at the detector from the reconstructed fields;
 *     E^n = E^{n+1} - cb (curl Ht^{n+1/2} - J) on the interior;
 *     grad += -lam_E . (E^{n+1} - E^n) / eps on the design box;
 *     transpose of the E half-step on lam (full grid, CPML included);
 *     restore E^n on the high layers (knots: samples and E^0 = 0 at time 0);
 *     Ht^{n-1/2} = Ht^{n+1/2} + S curl E^n on the interior;
 *     transpose of the H half-step on lam.
 * Cells outside the interior and the restored layers are set to NaN after
 * the forward run, so any use of a value the method does not have shows up.
 * fmt < 0 keeps the samples unquantised (exact FP64).
 */
int oracle_reverse2(const ocfg* c, const double* eps, int fmt, int scaled, int coeffs, int k,
                    int interp, double seed, double seed2, double* grad, double* obj2,
                    double* tape_values_out) {
  size_t N = ncell(c);
  const ocfg c2 = second_detector(c);
  int T = c->n_steps;
  if (k < 1 || T < 1 || c->P < 1) return -1;
  int r = (T - 1) % k;
  int J = (T - 1 - r) / k + 1;
  size_t ns = oracle_sample_values(c);
  int dX = c->dhi[0] - c->dlo[0], dY = c->dhi[1] - c->dlo[1], dZ = c->dhi[2] - c->dlo[2];
  size_t nd = (size_t)dX * dY * dZ;
  octx x;
  if (ctx_init(&x, c)) { ctx_free(&x); return -2; }
  double* st = (double*)calloc(NF * N, sizeof(double));
  double* lam = (double*)calloc(NF * N, sizeof(double));
  double* tmp = (double*)malloc(6 * N * sizeof(double));
  double* dE = (double*)calloc(3 * N, sizeof(double));
  double* tape = (double*)malloc((size_t)J * ns * sizeof(double));
  double* tk = (double*)malloc((size_t)(J + 1) * sizeof(double));
  double* pv = (double*)malloc((size_t)(J + 1) * sizeof(double));
  double* fb = (double*)malloc(ns * sizeof(double));
  if (!st || !lam || !tmp || !dE || !tape || !tk || !pv || !fb) {
    free(st); free(lam); free(tmp); free(dE); free(tape); free(tk); free(pv); free(fb);
    ctx_free(&x);
    return -2;
  }
  size_t foff[7]; foff[0] = 0;
  for (int f = 0; f < 6; ++f) foff[f + 1] = foff[f] + face_values(c, f);

  /* forward with recording */
  double L = 0.0, M = 0.0;
  for (int n = 0; n < T; ++n) {
    int sample = n >= r && (n - r) % k == 0;
    int j = (n - r) / k;
    if (sample)   /* E^n on the high faces, before the E update of step n */
      for (int f = 1; f < 6; f += 2) face_io(c, f, st, tape + (size_t)j * ns + foff[f], 0);
    h_update(&x, st);
    if (sample)   /* Ht^{n+1/2} on the low faces */
      for (int f = 0; f < 6; f += 2) face_io(c, f, st, tape + (size_t)j * ns + foff[f], 0);
    e_update(&x, eps, st, n);
    L += objective(c, st);
    if (c->det2_kind) M += objective(&c2, st);
  }
  if (fmt == 9) {   /* block-transform codec, K = coeffs (0: 10) */
    for (int j = 0; j < J; ++j)
      for (int f = 0; f < 6; ++f) {
        int ua, va, nu, nv; face_dims(c, f, &ua, &va, &nu, &nv);
        if (bdct_face(tape + (size_t)j * ns + foff[f], nu, nv, coeffs ? coeffs : 10)) {
          free(st); free(lam); free(tmp); free(dE); free(tape); free(tk); free(pv); free(fb);
          ctx_free(&x);
          return -2;
        }
      }
  } else if (fmt >= 0) {
    for (int j = 0; j < J; ++j)
      for (int f = 0; f < 6; ++f)
        encode_face(fmt, scaled, tape + (size_t)j * ns + foff[f], foff[f + 1] - foff[f], NULL);
  }
  if (tape_values_out) memcpy(tape_values_out, tape, (size_t)J * ns * sizeof(double));

  /* keep only what the method has: the interior of E and Ht */
  {
    int P = c->P;
    for (int f = 0; f < 6; ++f)
      for (int kk = 0; kk < c->nz; ++kk)
        for (int jj = 0; jj < c->ny; ++jj)
          for (int ii = 0; ii < c->nx; ++ii) {
            int in = ii >= P && ii < c->nx - P && jj >= P && jj < c->ny - P && kk >= P &&
                     kk < c->nz - P;
            if (!in) st[f * N + idx(c, ii, jj, kk)] = NAN;
          }
    for (size_t q = OFF_PSI * N; q < NF * N; ++q) st[q] = NAN;
  }

  for (size_t q = 0; q < nd; ++q) grad[q] = 0.0;
  for (int n = T - 1; n >= 0; --n) {
    /* restore Ht^{n+1/2}: knots -1 (zero) and s_j */
    int nk = 0;
    tk[nk++] = -1.0;
    for (int j = 0; j < J; ++j) tk[nk++] = r + (double)j * k;
    for (int f = 0; f < 6; f += 2) {
      for (size_t q = 0; q < foff[f + 1] - foff[f]; ++q) {
        pv[0] = 0.0;
        for (int j = 0; j < J; ++j) pv[1 + j] = tape[(size_t)j * ns + foff[f] + q];
        fb[foff[f] + q] = interp_eval(interp, tk, pv, nk, (double)n);
      }
      face_io(c, f, st, fb + foff[f], 1);
    }
    /* both detectors' adjoint sources, from the reconstructed (E^{n+1}, Ht^{n+1/2}) */
    objective_seed(c, st, seed, lam);
    if (c->det2_kind) objective_seed(&c2, st, seed2, lam);
    inverse_e(&x, eps, st, n, dE);
    grad_accumulate(c, eps, lam, dE, grad);
    adj_e_transpose(&x, eps, lam, tmp);
    /* restore E^n: knots 0 (zero, unless s_0 == 0) and s_j */
    nk = 0;
    if (r > 0) tk[nk++] = 0.0;
    for (int j = 0; j < J; ++j) tk[nk++] = r + (double)j * k;
    for (int f = 1; f < 6; f += 2) {
      for (size_t q = 0; q < foff[f + 1] - foff[f]; ++q) {
        int m = 0;
        if (r > 0) pv[m++] = 0.0;
        for (int j = 0; j < J; ++j) pv[m++] = tape[(size_t)j * ns + foff[f] + q];
        fb[foff[f] + q] = interp_eval(interp, tk, pv, nk, (double)n);
      }
      face_io(c, f, st, fb + foff[f], 1);
    }
    inverse_h(&x, st);
    adj_h_transpose(&x, lam, tmp);
  }
  if (obj2) { obj2[0] = L; obj2[1] = M; }
  free(st); free(lam); free(tmp); free(dE); free(tape); free(tk); free(pv); free(fb);
  ctx_free(&x);
  return 0;
}

/* The method for the first detector's objective alone (second detector ignored). */
int oracle_reverse_ex(const ocfg* c, const double* eps, int fmt, int scaled, int coeffs, int k,
                      int interp, double seed, double* grad, double* obj,
                      double* tape_values_out) {
  ocfg one = *c;
  one.det2_kind = 0;
  double o2[2];
  int rc = oracle_reverse2(&one, eps, fmt, scaled, coeffs, k, interp, seed, 0.0, grad, o2,
                           tape_values_out);
  if (obj) *obj = o2[0];
  return rc;
}

int oracle_reverse(const ocfg* c, const double* eps, int fmt, int scaled, int k, int interp,
                   double seed, double* grad, double* obj, double* tape_values_out) {
  return oracle_reverse_ex(c, eps, fmt, scaled, 0, k, interp, seed, grad, obj, tape_values_out);
}

/* ---------------------------------------- the method's pieces, exported ----
 * Single operations of the method above on the full grid, for tests that run
 * it piece by piece (for instance split into z slabs, each holding only its
 * own planes).  st and lam: NF arrays of ncell doubles.
 *   op 0: H half-step of the forward (st);
 *   op 1: E half-step of step n (st);
 *   op 2: inverse E half-step of step n on the interior (st); dE (3 ncell,
 *         optional) receives E^{n+1} - E^n there;
 *   op 3: inverse H half-step on the interior (st);
 *   op 4: transpose of the E half-step (lam; tmp: 6 ncell doubles);
 *   op 5: transpose of the H half-step (lam; tmp);
 *   op 6: grad += -lam_E . dE / eps on the design box (lam, dE, grad).
 */
int oracle_op(const ocfg* c, const double* eps, int op, int n, double* st, double* lam,
              double* tmp, double* dE, double* grad) {
  octx x;
  if (op < 0 || op > 6) return -1;
  if (ctx_init(&x, c)) { ctx_free(&x); return -2; }
  switch (op) {
    case 0: h_update(&x, st); break;
    case 1: e_update(&x, eps, st, n); break;
    case 2: inverse_e(&x, eps, st, n, dE); break;
    case 3: inverse_h(&x, st); break;
    case 4: adj_e_transpose(&x, eps, lam, tmp); break;
    case 5: adj_h_transpose(&x, lam, tmp); break;
    default: grad_accumulate(c, eps, lam, dE, grad); break;
  }
  ctx_free(&x);
  return 0;
}

/* l_n of the detector from the state (E^{n+1}, Ht^{n+1/2}). */
double oracle_objective(const ocfg* c, const double* st) {
  return c->det_kind ? objective(c, st) : 0.0;
}

/* lam += seed * dl_n / d(E^{n+1}, Ht^{n+1/2}) on the detector. */
void oracle_objective_seed(const ocfg* c, const double* st, double seed, double* lam) {
  if (c->det_kind) objective_seed(c, st, seed, lam);
}

/* Face f's interface layer: dir 0 copies state -> buf, dir 1 buf -> state
 * (values [tangential comp][v][u], the tape's order). */
int oracle_face_io(const ocfg* c, int f, double* st, double* buf, int dir) {
  if (f < 0 || f > 5 || c->P < 1) return -1;
  face_io(c, f, st, buf, dir);
  return 0;
}
