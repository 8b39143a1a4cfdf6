// fdtd_api.cu -- host side of the library: plan, workspace, orchestration, C ABI.
//
// A handle holds the plan of one problem (grid, CPML tables, source, detector,
// design box, step count) and, after fdtd_forward, the state the backward run
// starts from.  Device memory is the caller's workspace; the library creates
// only its own stream, events and CUDA graphs.  The time loops (hundreds to
// thousands of launches) are captured once per record configuration and
// replayed as CUDA graphs.
#include <limits.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/fdtd.h"
#include "bdct.cuh"
#include "fdtd_internal.cuh"

using namespace fdtd;

namespace {

const double kC0 = 299792458.0;

struct Layout {
  size_t F[3], L[2], cb, eps, psiF[2], psiL[2], gacc, gout, obj, obj2, seeds, prof, srcw, tape,
      scales, err;
  PsiLayout plF, plL;  // layouts of the forward and adjoint auxiliary sets
  size_t total;
  long long stride;   // tape elements per sample
  int J;              // samples
};

struct GraphKey {
  int dir, dtype, k, interp, scaled, kernel, tile_y, zchunk, sample, stages, pdl, prefetch,
      tile_x, compact, exact, coeffs, zchunk_fwd, zgroups, inject_wait, reverse, forward,
      zchunk_fwd2, start_buf;
  bool operator<(const GraphKey& o) const {
    return memcmp(this, &o, sizeof(GraphKey)) < 0;
  }
};

}  // namespace

// One sampled interval of a time loop: type 0 = a single launch of kind q,
// type 1 = two consecutive launches, kind p then kind q; -1 = left open.
struct SampleEntry {
  int type, p, q;
};

struct GraphEntry {
  cudaGraphExec_t exec;
  std::vector<SampleEntry> plan;   // intervals the graph's event nodes record
};

struct BatchPlan;

struct fdtd_handle {
  int nx, ny, nz, px, P, N, nmax;
  double S, dx, dt;
  fdtd_pml pml;
  fdtd_source src;
  fdtd_detector det;
  fdtd_detector det2;         // optional second detector (kind 0 = none)
  double seeds[2];            // backward seeds of the two detectors over seed_scale (host copy)
  double seed_scale;          // reference seed, applied when the gradient is finalised
  int dlo[3], dhi[3];
  cudaStream_t user_stream;

  std::vector<float> prof;    // [3][6][nmax]
  std::vector<float> wave;    // [N]
  std::vector<float> srcw;    // source weights over its region
  int src_u0, src_u1, src_v0, src_v1, src_axis, src_index;
  Faces faces;

  char* ws;
  size_t ws_bytes;
  bool tables_uploaded;
  bool have_forward;
  int fwd_buf;                // field buffer holding the state after forward
  fdtd_record_cfg fwd_rec;

  int opt_graphs, opt_kernel, opt_tile_y, opt_zchunk, opt_sample, opt_stages, opt_pdl,
      opt_prefetch, opt_tile_x, opt_compact, opt_exact, opt_zchunk_fwd, opt_zgroups,
      opt_zchunk_fwd2;
  int opt_inject_wait;        // FDTD_OPT_INJECT_WAIT_TIMEOUT (SM cycles; 0 = off)
  int opt_reverse;            // FDTD_OPT_REVERSE: 0 automatic, 1 split phases, 2 fused
  int opt_forward;            // FDTD_OPT_FORWARD: 0 automatic, 1 split half-steps, 2 fused,
                              // 3 two steps per pass
  // z-group scheduling (FDTD_OPT_ZGROUPS): one stream per group, and per group
  // three events (the last launch of an even / odd phase, the join), plus the
  // fork event
  std::vector<cudaStream_t> zs;
  std::vector<cudaEvent_t> zev;
  cudaEvent_t zfork;
  // sampled kernel timing (see Sampler): per direction a pool of start / end
  // events and the intervals the last enqueued or replayed loop recorded
  std::vector<cudaEvent_t> spool[2][2];
  std::vector<SampleEntry> splan[2];
  float savg[FDTD_K_KINDS];
  int scount[FDTD_K_KINDS];

  cudaStream_t stream;
  cudaEvent_t ev_in, ev_out, t0, t1, t2, t3, t4, t5;
  float host_call_ms;         // device part of the last fdtd_value_and_grad_host
  bool cuda_ready;
  std::map<GraphKey, GraphEntry> graphs;
  int launches_fwd, launches_bwd;
  float fwd_ms, bwd_ms;
  std::vector<double> obj_hist;
  double obj2_sum;            // second detector's objective of the last forward
  BatchPlan* batch;           // batched-designs plan led by this handle (fdtd_batch_*)
  std::string err;
};

static void drop_batch(fdtd_handle* h);

static const int kMaxZGroups = 16;
static std::string g_create_error;

static int fail(fdtd_handle* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  else g_create_error = msg;
  return code;
}

static int cuda_fail(fdtd_handle* h, const char* what, cudaError_t e) {
  char buf[256];
  snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
  return fail(h, FDTD_ECUDA, buf);
}

#define CK(h, x)                                   \
  do {                                             \
    cudaError_t e_ = (x);                          \
    if (e_ != cudaSuccess) return cuda_fail(h, #x, e_); \
  } while (0)

// ------------------------------------------------------------ CPML plan ---
// Depth into the absorbing layer of a derivative at coordinate x (cells; E
// derivatives at integers, H derivatives at half-integers).  The lossless
// span [P, N-P-1/2] holds every E and H position of the interior cells, so
// the interior update has no CPML terms and can be inverted exactly.
static double layer_depth(int n, int P, double x) {
  double lo = (double)P, hi = (double)(n - P) - 0.5;
  double cells = 0.0;
  if (x < lo) cells = lo - x;
  else if (x > hi) cells = x - hi;
  return cells / P;
}

static void cpml_coeffs(const fdtd_handle* h, double d, float out[3]) {
  if (d <= 0.0) {
    out[0] = 0.f;
    out[1] = 0.f;
    out[2] = 1.f;
    return;
  }
  const double m = h->pml.order;
  const double grade = pow(d, m);
  const double sigma = h->pml.sigma_factor * (m + 1.0) * h->S * grade;  // sigma dt / eps0
  const double kappa = 1.0 + (h->pml.kappa_max - 1.0) * grade;
  const double w0dt = 2.0 * M_PI * h->S * h->dx / h->src.lambda0;      // 2 pi f0 dt
  const double alpha = h->pml.alpha_factor * w0dt * (1.0 - d);          // alpha dt / eps0
  const double b = exp(-(sigma / kappa + alpha));
  const double a = sigma * (b - 1.0) / (kappa * (sigma + kappa * alpha));
  out[0] = (float)b;
  out[1] = (float)a;
  out[2] = (float)(1.0 / kappa);
}

static void build_profiles(fdtd_handle* h) {
  int dims[3] = {h->nx, h->ny, h->nz};
  h->prof.assign(3 * 6 * h->nmax, 0.f);
  for (int ax = 0; ax < 3; ++ax) {
    for (int i = 0; i < dims[ax]; ++i) {
      float e[3], hh[3];
      cpml_coeffs(h, layer_depth(dims[ax], h->P, (double)i), e);
      cpml_coeffs(h, layer_depth(dims[ax], h->P, (double)i + 0.5), hh);
      for (int w = 0; w < 3; ++w) {
        h->prof[(ax * 6 + w) * h->nmax + i] = e[w];
        h->prof[(ax * 6 + 3 + w) * h->nmax + i] = hh[w];
      }
    }
  }
}

// ---------------------------------------------------------------- source ---
// Gaussian-modulated carrier sampled at the half steps; times in units of dt.
static void build_source(fdtd_handle* h) {
  h->wave.assign(h->N, 0.f);
  h->srcw.clear();
  const fdtd_source& s = h->src;
  if (s.kind == FDTD_SRC_NONE) return;
  const double w0 = 2.0 * M_PI * h->S * h->dx / s.lambda0;  // rad per step
  const double tau = 2.0 * sqrt(2.0 * M_LN2) / (s.rel_bandwidth * w0);
  const double t0 = s.t0_over_tau * tau;
  for (int n = 0; n < h->N; ++n) {
    double t = (n + 0.5) - t0;
    double env = exp(-(t * t) / (tau * tau));
    h->wave[n] = (float)(s.amplitude * env * sin(w0 * t));
  }
  int dims[3] = {h->nx, h->ny, h->nz};
  if (s.kind == FDTD_SRC_POINT) {
    h->src_axis = 2;
    h->src_index = s.pos[2];
    h->src_u0 = s.pos[0];
    h->src_u1 = s.pos[0] + 1;
    h->src_v0 = s.pos[1];
    h->src_v1 = s.pos[1] + 1;
    h->srcw.assign(1, 1.f);
  } else {
    int a = s.axis, ua = a == 0 ? 1 : 0, va = a == 2 ? 1 : 2;
    h->src_axis = a;
    h->src_index = s.pos[a];
    h->src_u0 = h->P;
    h->src_u1 = dims[ua] - h->P;
    h->src_v0 = h->P;
    h->src_v1 = dims[va] - h->P;
    int nu = h->src_u1 - h->src_u0, nv = h->src_v1 - h->src_v0;
    h->srcw.resize((size_t)nu * nv);
    for (int v = 0; v < nv; ++v)
      for (int u = 0; u < nu; ++u) {
        double ru = (h->src_u0 + u - s.pos[ua]) / s.sigma_uv[0];
        double rv = (h->src_v0 + v - s.pos[va]) / s.sigma_uv[1];
        h->srcw[(size_t)v * nu + u] =
            s.kind == FDTD_SRC_PLANE_UNIFORM ? 1.f : (float)exp(-0.5 * (ru * ru + rv * rv));
      }
  }
}

// ----------------------------------------------------------------- faces ---
static void build_faces(fdtd_handle* h) {
  int dims[3] = {h->nx, h->ny, h->nz};
  int start = 0;
  h->faces.start[0] = 0;
  for (int f = 0; f < 6; ++f) {
    FaceDesc& d = h->faces.f[f];
    int a = f / 2, high = f & 1;
    d.axis = a;
    d.ua = a == 0 ? 1 : 0;
    d.va = a == 2 ? 1 : 2;
    d.nu = dims[d.ua] - 2 * h->P;
    d.nv = dims[d.va] - 2 * h->P;
    d.layer = high ? dims[a] - h->P : h->P - 1;
    int base = high ? 0 : 3;  // E on high faces, Ht on low faces
    d.comp0 = base + d.ua;
    d.comp1 = base + d.va;
    d.off = start;
    start += 2 * d.nu * d.nv;
    h->faces.start[f + 1] = start;
  }
}

static long long sample_elems(const fdtd_handle* h) { return h->faces.start[6]; }

static int n_samples(int N, int k) {
  int r = (N - 1) % k;
  return (N - 1 - r) / k + 1;
}

static bool valid_dtype(int dt) { return (dt >= 0 && dt < kTapeDtypes) || dt == kTapeBdct; }
// coeffs: 0..64 for BDCT (0 = the default), 0 for every other type.
static bool coeffs_ok(const fdtd_record_cfg* rec) {
  return rec->dtype == kTapeBdct ? rec->coeffs >= 0 && rec->coeffs <= 64 : rec->coeffs == 0;
}
static int bdct_coeffs(const fdtd_record_cfg* rec) {
  return rec->coeffs ? rec->coeffs : kBdctDefaultCoeffs;
}

// Bytes of one tape sample (padded to 16) and the element size its offsets
// count in.
static long long sample_bytes(const fdtd_handle* h, const fdtd_record_cfg* rec) {
  if (rec && rec->dtype == kTapeBdct) return bdct_layout(h->faces, bdct_coeffs(rec)).sample_bytes;
  const int eb = code_bytes(rec ? rec->dtype : 0);
  return (sample_elems(h) * eb + 15) / 16 * 16;
}

// ---------------------------------------------------------- interpolation ---
// Knots of the recorded series in step units: samples at r + j k and the
// known zero initial state (Ht^{-1/2} at -1; E^0 at 0 unless 0 is a sample).
// The value at step n is sum_m weight_m * sample(slot_m): linear uses the two
// bracketing knots; cubic is a cubic Hermite whose knot slopes are those of
// the Lagrange quadratic through the knot and its neighbours (one-sided at
// the ends), i.e. Catmull-Rom on evenly spaced knots.
struct Knots {
  std::vector<double> t;
  std::vector<int> slot;  // -1 for the zero knot
};

static Knots make_knots(int N, int k, int field) {
  Knots K;
  int r = (N - 1) % k;
  int J = n_samples(N, k);
  if (field == 0) {
    K.t.push_back(-1.0);
    K.slot.push_back(-1);
  } else if (r > 0) {
    K.t.push_back(0.0);
    K.slot.push_back(-1);
  }
  for (int j = 0; j < J; ++j) {
    K.t.push_back((double)(r + j * k));
    K.slot.push_back(j);
  }
  return K;
}

// Derivative weights at node x of the quadratic through nodes (a, b, c):
// d/dx of the Lagrange basis polynomials.
static void lagrange_slope(double a, double b, double c, double x, double w[3]) {
  w[0] = ((x - b) + (x - c)) / ((a - b) * (a - c));
  w[1] = ((x - a) + (x - c)) / ((b - a) * (b - c));
  w[2] = ((x - a) + (x - b)) / ((c - a) * (c - b));
}

// Slope at knot j as weights over knot indices idx[0..2].
static void knot_slope(const Knots& K, int j, int idx[3], double w[3]) {
  int n = (int)K.t.size();
  if (n == 2) {
    idx[0] = 0; idx[1] = 1; idx[2] = 1;
    double h = K.t[1] - K.t[0];
    w[0] = -1.0 / h; w[1] = 1.0 / h; w[2] = 0.0;
    return;
  }
  int c = j;
  if (c < 1) c = 1;
  if (c > n - 2) c = n - 2;
  idx[0] = c - 1; idx[1] = c; idx[2] = c + 1;
  lagrange_slope(K.t[c - 1], K.t[c], K.t[c + 1], K.t[j], w);
}

static void interp_weights(const fdtd_handle* h, const fdtd_record_cfg* rec, int n, int field,
                           int slot[4], float wt[4]) {
  for (int m = 0; m < 4; ++m) { slot[m] = -1; wt[m] = 0.f; }
  Knots K = make_knots(h->N, rec->k, field);
  int nk = (int)K.t.size();
  double q = (double)n;
  int a = 0;
  while (a + 1 < nk && K.t[a + 1] < q) ++a;
  // exact knot hit
  for (int j = 0; j < nk; ++j)
    if (K.t[j] == q) {
      slot[0] = K.slot[j];
      wt[0] = 1.f;
      return;
    }
  if (a + 1 >= nk) { slot[0] = K.slot[nk - 1]; wt[0] = 1.f; return; }
  int b = a + 1;
  double hh = K.t[b] - K.t[a];
  double s = (q - K.t[a]) / hh;
  std::map<int, double> acc;  // knot index -> weight
  if (rec->interp == FDTD_INTERP_LINEAR || nk < 2) {
    acc[a] += 1.0 - s;
    acc[b] += s;
  } else {
    double h00 = (1 + 2 * s) * (1 - s) * (1 - s), h10 = s * (1 - s) * (1 - s);
    double h01 = s * s * (3 - 2 * s), h11 = -s * s * (1 - s);
    acc[a] += h00;
    acc[b] += h01;
    int ia[3], ib[3];
    double wa[3], wb[3];
    knot_slope(K, a, ia, wa);
    knot_slope(K, b, ib, wb);
    for (int m = 0; m < 3; ++m) {
      acc[ia[m]] += h10 * hh * wa[m];
      acc[ib[m]] += h11 * hh * wb[m];
    }
  }
  int m = 0;
  for (auto& kv : acc) {
    if (K.slot[kv.first] < 0 || kv.second == 0.0) continue;  // zero knot contributes nothing
    if (m < 4) {
      slot[m] = K.slot[kv.first];
      wt[m] = (float)kv.second;
      ++m;
    }
  }
}

// The reverse step of kernel 5 runs as two fused launches (primal and
// adjoint, kernels_rev_fused.cu) unless FDTD_OPT_REVERSE asks for the split
// phases; the fused kernels are built for 32 x 8 tiles.
// Automatic (0): fused where at most half of the (tile, chunk) units carry
// CPML terms, which its adjoint evaluates in a heavier variant (measured on
// GB300: the reverse 11 % faster than split on 600 x 600 x 300 with 31 % of
// the units in the CPML, 28 % slower on 200 x 200 x 100 with 70 %).
static bool fused_reverse(const fdtd_handle* h) {
  if (h->opt_kernel != 5 || h->opt_reverse == 1) return false;
  const int ty = h->opt_tile_y < 2 ? 2 : h->opt_tile_y;
  const int tx = (ty == 8 && h->opt_stages <= 3 && h->opt_tile_x == 40) ? 40 : 32;
  if (ty != 8 || tx != 32) return false;
  if (h->opt_reverse == 2) return true;
  Geo g;
  memset(&g, 0, sizeof g);
  g.nx = h->nx; g.ny = h->ny; g.nz = h->nz; g.P = h->P;
  const RevUnits U = rev_units(g, h->opt_zchunk > 0 ? h->opt_zchunk : h->nz);
  const long long all = (long long)U.ntx * U.nty * U.nzc;
  const long long cpml = all - (long long)(U.ix1 - U.ix0) * (U.iy1 - U.iy0) * (U.iz1 - U.iz0);
  return 2 * cpml <= all;
}

// Planes per z chunk of a fused forward step (the unit grid of its launches).
static int fused_forward_zchunk(const fdtd_handle* h) {
  if (h->opt_zchunk_fwd > 0) return h->opt_zchunk_fwd;
  return h->opt_zchunk > 0 ? h->opt_zchunk : h->nz;
}

// Does the plane region (normal `axis` at `index`, [u0, u1) x [v0, v1) in the
// other two axes, increasing axis order) meet the cell box [lo, hi)?
static bool plane_meets(int axis, int index, int u0, int u1, int v0, int v1, const int lo[3],
                        const int hi[3]) {
  const int ua = axis == 0 ? 1 : 0, va = axis == 2 ? 1 : 2;
  return index >= lo[axis] && index < hi[axis] && u0 < hi[ua] && u1 > lo[ua] && v0 < hi[va] &&
         v1 > lo[va];
}

// The forward step of kernel 5 runs the units without a CPML term as one
// fused launch (both half-steps, kernels_fwd_fused.cu) and the other units
// with the split half-steps, unless FDTD_OPT_FORWARD asks for the split
// half-steps everywhere.  It needs 32 x 8 tiles, such units, and the source
// and the detector outside them (the split E half-step adds the source and
// sums the objective).  Automatic (0): as the reverse step, fused where at
// most half of the units carry CPML terms, unless the two-step pass (below)
// runs there.
static bool two_step_forward(const fdtd_handle* h);

static bool fused_forward(const fdtd_handle* h) {
  if (h->opt_kernel != 5 || h->opt_forward == 1 || h->opt_forward == 3) return false;
  if (h->opt_forward == 0 && two_step_forward(h)) return false;   // automatic: two steps per pass
  const int ty = h->opt_tile_y < 2 ? 2 : h->opt_tile_y;
  const int tx = (ty == 8 && h->opt_stages <= 3 && h->opt_tile_x == 40) ? 40 : 32;
  if (ty != 8 || tx != 32) return false;
  Geo g;
  memset(&g, 0, sizeof g);
  g.nx = h->nx; g.ny = h->ny; g.nz = h->nz; g.P = h->P;
  const int zc = fused_forward_zchunk(h);
  const RevUnits U = rev_units(g, zc);
  if (U.ix1 <= U.ix0 || U.iy1 <= U.iy0 || U.iz1 <= U.iz0) return false;
  const int lo[3] = {U.ix0 * 32, U.iy0 * 8, U.iz0 * zc};
  const int hi[3] = {U.ix1 * 32, U.iy1 * 8, std::min(U.iz1 * zc, h->nz)};
  if (h->src.kind && plane_meets(h->src_axis, h->src_index, h->src_u0, h->src_u1, h->src_v0,
                                 h->src_v1, lo, hi))
    return false;
  if (h->det.kind && plane_meets(h->det.axis, h->det.index, h->det.lo[0], h->det.hi[0],
                                 h->det.lo[1], h->det.hi[1], lo, hi))
    return false;
  if (h->opt_forward == 2) return true;
  const long long all = (long long)U.ntx * U.nty * U.nzc;
  const long long cpml = all - (long long)(U.ix1 - U.ix0) * (U.iy1 - U.iy0) * (U.iz1 - U.iz0);
  return 2 * cpml <= all;
}

// Two time steps per pass (kernels_fwd_2step.cu, FDTD_OPT_FORWARD = 3): the
// deep units run steps n and n + 1 in one launch, the other units the split
// half-steps one step at a time through a third field buffer.  Needs kernel
// 5 with 32 x 8 tiles, deep units, and the source and the detectors at least
// two cells away from the deep box (the pass evaluates the intermediate
// level on a two-cell halo and adds no source term, sums no objective).
// Automatic (0): where the fused step would run (at most half of the units
// carry CPML terms), which it beats on 600 x 600 x 300 (1028 against 1166 us
// per forward step); on 200 x 200 x 100 it is slower than the split
// half-steps (92 against 59 us), as the fused step is.
static bool two_step_forward(const fdtd_handle* h) {
  if (h->opt_kernel != 5 || (h->opt_forward != 3 && h->opt_forward != 0)) return false;
  const int ty = h->opt_tile_y < 2 ? 2 : h->opt_tile_y;
  const int tx = (ty == 8 && h->opt_stages <= 3 && h->opt_tile_x == 40) ? 40 : 32;
  if (ty != 8 || tx != 32) return false;
  Geo g;
  memset(&g, 0, sizeof g);
  g.nx = h->nx; g.ny = h->ny; g.nz = h->nz; g.P = h->P;
  const int zc = fused_forward_zchunk(h);
  const RevUnits U = deep_units(g, zc);
  if (U.ix1 <= U.ix0 || U.iy1 <= U.iy0 || U.iz1 <= U.iz0) return false;
  const int lo[3] = {U.ix0 * 32 - 2, U.iy0 * 8 - 2, U.iz0 * zc - 2};
  const int hi[3] = {U.ix1 * 32 + 2, U.iy1 * 8 + 2, std::min(U.iz1 * zc, h->nz) + 2};
  if (h->src.kind && plane_meets(h->src_axis, h->src_index, h->src_u0, h->src_u1, h->src_v0,
                                 h->src_v1, lo, hi))
    return false;
  if (h->det.kind && plane_meets(h->det.axis, h->det.index, h->det.lo[0], h->det.hi[0],
                                 h->det.lo[1], h->det.hi[1], lo, hi))
    return false;
  if (h->det2.kind && plane_meets(h->det2.axis, h->det2.index, h->det2.lo[0], h->det2.hi[0],
                                  h->det2.lo[1], h->det2.hi[1], lo, hi))
    return false;
  if (h->opt_forward == 3) return true;
  const RevUnits R = rev_units(g, zc);
  const long long all = (long long)R.ntx * R.nty * R.nzc;
  const long long cpml = all - (long long)(R.ix1 - R.ix0) * (R.iy1 - R.iy0) * (R.iz1 - R.iz0);
  return R.ix1 > R.ix0 && 2 * cpml <= all;
}

// The field buffer holding the state after a forward: the fused step flips
// the pair every step, the two-step pass every pair of steps (and its split
// first step, for an odd count, once).
static int forward_end_buf(const fdtd_handle* h) {
  if (two_step_forward(h)) return ((h->N + 1) / 2) & 1;
  return fused_forward(h) ? (h->N & 1) : 0;
}

// ---------------------------------------------------------------- layout ---
static size_t al(size_t x) { return (x + 255) & ~(size_t)255; }
static int rup4(int x) { return (x + 3) & ~3; }

// Auxiliary-set layout.  Full: every axis array spans the grid (the layout
// of the older kernels, component c of axis a at (4a + c) nc).  Compact
// (two-cells-per-thread kernels only): the array of axis a holds only the
// cells of a's two slabs, per axis where the grid is long enough that no
// staged box reaches both slabs: along x the low part keeps [0, Wlo) and the
// high slab starts at the 4-aligned cell hs, so that box starts stay on
// 16-byte boundaries; along y and z the high slab follows the low one.
static PsiLayout psi_layout(const fdtd_handle* h, bool compact) {
  PsiLayout pl;
  const int P = h->P;
  long long off = 0;
  for (int a = 0; a < 3; ++a) {
    PsiAxis& A = pl.ax[a];
    A.d0 = h->px; A.e0 = h->nx; A.d1 = h->ny; A.d2 = h->nz;
    A.hs = INT_MAX; A.shift = 0;
    if (compact && a == 0 && h->nx >= 2 * P + 56) {
      const int wlo = rup4(P), hs = (h->nx - P) & ~3;
      A.hs = hs; A.shift = hs - wlo;
      A.e0 = wlo + (h->nx - hs);
      A.d0 = rup4(A.e0);
    } else if (compact && a == 1 && h->ny >= 2 * P + 24) {
      A.hs = h->ny - P; A.shift = h->ny - 2 * P; A.d1 = 2 * P;
    } else if (compact && a == 2 && h->nz >= 2 * P + 1) {
      A.hs = h->nz - P; A.shift = h->nz - 2 * P; A.d2 = 2 * P;
    }
    A.ps = (long long)A.d0 * A.d1;
    A.cs = A.ps * A.d2;
    A.off = off;
    off += 4 * A.cs;
  }
  pl.total = off;
  return pl;
}

static Layout layout_of(const fdtd_handle* h, const fdtd_record_cfg* rec) {
  Layout L;
  size_t nc = (size_t)h->nz * h->ny * h->px;
  size_t f6 = al(6 * nc * sizeof(float));
  // the staged kernels (5) keep their auxiliaries compact
  L.plF = psi_layout(h, h->opt_compact && h->opt_kernel == 5);
  L.plL = psi_layout(h, h->opt_compact && h->opt_kernel == 5);
  size_t psbF = al((size_t)L.plF.total * sizeof(float));
  size_t psbL = al((size_t)L.plL.total * sizeof(float));
  size_t nd = (size_t)(h->dhi[0] - h->dlo[0]) * (h->dhi[1] - h->dlo[1]) * (h->dhi[2] - h->dlo[2]);
  // the fused steps write the new fields (and, in reverse, adjoint fields)
  // next to the old ones (ping-pong pairs)
  const bool rev2 = fused_reverse(h), fwd2 = fused_forward(h), two = two_step_forward(h);
  size_t off = 0;
  L.F[0] = off; off += f6;
  L.F[1] = L.F[0];
  if (rev2 || fwd2 || two) { L.F[1] = off; off += f6; }
  L.F[2] = L.F[0];
  if (two) { L.F[2] = off; off += f6; }   // the two-step pass's intermediate level
  L.L[0] = off; off += f6;
  L.L[1] = L.L[0];
  if (rev2) { L.L[1] = off; off += f6; }
  L.cb = off; off += al(nc * sizeof(float));
  L.eps = off; off += al((size_t)h->nx * h->ny * h->nz * sizeof(float));
  L.psiF[0] = off; off += psbF;
  L.psiF[1] = L.psiF[0];
  L.psiL[0] = off; off += psbL;
  L.psiL[1] = off; off += psbL;
  L.gacc = off; off += al(nd * sizeof(double));
  L.gout = off; off += al(nd * sizeof(float));
  L.obj = off; off += al((size_t)h->N * sizeof(double));
  L.obj2 = off; off += al((size_t)h->N * sizeof(double));
  L.seeds = off; off += al(2 * sizeof(double));
  L.prof = off; off += al(h->prof.size() * sizeof(float));
  L.srcw = off; off += al((h->srcw.size() + 1) * sizeof(float));
  L.err = off; off += 256;
  int dt = rec ? rec->dtype : 0;
  int k = rec ? rec->k : 1;
  int eb = dt == kTapeBdct ? 1 : code_bytes(dt);
  long long stride = sample_bytes(h, rec) / eb;
  L.stride = stride;
  L.J = n_samples(h->N, k);
  L.tape = off; off += al((size_t)L.J * stride * eb);
  L.scales = off; off += al((size_t)L.J * 6 * sizeof(float));
  L.total = off;
  return L;
}

static Geo geo_of(const fdtd_handle* h) {
  Geo g;
  g.nx = h->nx; g.ny = h->ny; g.nz = h->nz; g.px = h->px; g.P = h->P; g.nmax = h->nmax;
  g.plane = (long long)h->ny * h->px;
  g.nc = (long long)h->nz * g.plane;
  g.S = (float)h->S;
  g.prof = nullptr;
  return g;
}

static int check_rec(fdtd_handle* h, const fdtd_record_cfg* rec) {
  if (!rec) return fail(h, FDTD_EINVAL, "record config is NULL");
  if (!valid_dtype(rec->dtype)) return fail(h, FDTD_EINVAL, "unknown tape dtype");
  if (rec->k < 1) return fail(h, FDTD_EINVAL, "k must be >= 1");
  if (rec->interp != FDTD_INTERP_LINEAR && rec->interp != FDTD_INTERP_CUBIC)
    return fail(h, FDTD_EINVAL, "unknown interpolation");
  if (rec->scaled && (rec->dtype < 2 || rec->dtype == kTapeBdct))
    return fail(h, FDTD_EINVAL, "per-face scale applies to F16 and the 8-bit types only");
  if (!coeffs_ok(rec)) return fail(h, FDTD_EINVAL, "coeffs: 0..64 for BDCT, 0 otherwise");
  return FDTD_OK;
}

// ------------------------------------------------------------- create ---
static const char* detector_error(const fdtd_detector& det, const int dims[3], int P) {
  if (det.kind == 0) return nullptr;
  if (det.kind != FDTD_OBJ_E2_PLANE && det.kind != FDTD_OBJ_POYNTING_PLANE)
    return "unknown detector kind";
  if (det.axis < 0 || det.axis > 2) return "detector axis 0..2";
  int ua = det.axis == 0 ? 1 : 0, va = det.axis == 2 ? 1 : 2;
  if (det.index < P || det.index >= dims[det.axis] - P)
    return "detector plane must be inside the interior";
  if (det.lo[0] < P || det.hi[0] > dims[ua] - P || det.lo[0] >= det.hi[0] || det.lo[1] < P ||
      det.hi[1] > dims[va] - P || det.lo[1] >= det.hi[1])
    return "detector window must be non-empty and inside the interior";
  return nullptr;
}

extern "C" int fdtd_create(const fdtd_grid* grid, double dx, double dt, const fdtd_pml* pml,
                           const fdtd_source* source, const fdtd_detector* detector, int n_steps,
                           const int design_lo[3], const int design_hi[3], void* cuda_stream,
                           fdtd_handle** out) {
  if (!out) return fail(nullptr, FDTD_EINVAL, "out is NULL");
  *out = nullptr;
  if (!grid || !pml || !design_lo || !design_hi)
    return fail(nullptr, FDTD_EINVAL, "NULL argument");
  int P = pml->thickness;
  int dims[3] = {grid->nx, grid->ny, grid->nz};
  if (P < 1) return fail(nullptr, FDTD_EINVAL, "PML thickness must be >= 1");
  for (int a = 0; a < 3; ++a)
    if (dims[a] < 2 * P + 2 || dims[a] > (1 << 20))
      return fail(nullptr, FDTD_EINVAL, "each grid size must be >= 2*P+2");
  if (!(dx > 0) || !(dt > 0)) return fail(nullptr, FDTD_EINVAL, "dx and dt must be > 0");
  double S = kC0 * dt / dx;
  if (S > 1.0 / sqrt(3.0) * (1.0 + 1e-12))
    return fail(nullptr, FDTD_EINVAL, "c dt / dx exceeds the 3D CFL limit 1/sqrt(3) (Eq. 1)");
  if (n_steps < 1) return fail(nullptr, FDTD_EINVAL, "n_steps must be >= 1");
  for (int a = 0; a < 3; ++a)
    if (design_lo[a] < P || design_hi[a] > dims[a] - P || design_lo[a] >= design_hi[a])
      return fail(nullptr, FDTD_EINVAL, "design box must be non-empty and inside the interior");
  fdtd_source src = {};
  if (source) src = *source;
  if (src.kind != FDTD_SRC_NONE) {
    if (src.kind != FDTD_SRC_POINT && src.kind != FDTD_SRC_PLANE_GAUSS &&
        src.kind != FDTD_SRC_PLANE_UNIFORM)
      return fail(nullptr, FDTD_EINVAL, "unknown source kind");
    if (src.component < 0 || src.component > 2)
      return fail(nullptr, FDTD_EINVAL, "source component must be 0..2");
    if (!(src.lambda0 > 0) || !(src.rel_bandwidth > 0))
      return fail(nullptr, FDTD_EINVAL, "source lambda0 and bandwidth must be > 0");
    if (src.kind == FDTD_SRC_POINT) {
      for (int a = 0; a < 3; ++a)
        if (src.pos[a] < P || src.pos[a] >= dims[a] - P)
          return fail(nullptr, FDTD_EINVAL, "point source must be inside the interior");
    } else {
      if (src.axis < 0 || src.axis > 2)
        return fail(nullptr, FDTD_EINVAL, "source axis must be 0..2");
      if (src.pos[src.axis] < P || src.pos[src.axis] >= dims[src.axis] - P)
        return fail(nullptr, FDTD_EINVAL, "source plane must be inside the interior");
      if (src.kind == FDTD_SRC_PLANE_GAUSS && (!(src.sigma_uv[0] > 0) || !(src.sigma_uv[1] > 0)))
        return fail(nullptr, FDTD_EINVAL, "source widths must be > 0");
    }
  } else {
    src.lambda0 = 1550e-9;  // sets alpha of the CPML only
  }
  fdtd_detector det = {};
  if (detector) det = *detector;
  if (const char* msg = detector_error(det, dims, P)) return fail(nullptr, FDTD_EINVAL, msg);
  fdtd_handle* h = new (std::nothrow) fdtd_handle();
  if (!h) return fail(nullptr, FDTD_ENOMEM, "host allocation failed");
  h->nx = dims[0]; h->ny = dims[1]; h->nz = dims[2];
  h->px = (h->nx + 7) & ~7;
  h->P = P;
  h->N = n_steps;
  h->nmax = std::max(h->nx, std::max(h->ny, h->nz));
  h->S = S; h->dx = dx; h->dt = dt;
  h->pml = *pml;
  if (h->pml.order <= 0) h->pml.order = 3;
  if (h->pml.sigma_factor < 0) h->pml.sigma_factor = 0.8;
  if (h->pml.kappa_max <= 0) h->pml.kappa_max = 1.0;
  if (h->pml.alpha_factor < 0) h->pml.alpha_factor = 0.05;
  h->src = src;
  h->det = det;
  h->det2 = fdtd_detector{};
  h->seeds[0] = 1.0;
  h->seeds[1] = 0.0;
  h->seed_scale = 1.0;
  h->obj2_sum = 0.0;
  for (int a = 0; a < 3; ++a) { h->dlo[a] = design_lo[a]; h->dhi[a] = design_hi[a]; }
  h->user_stream = (cudaStream_t)cuda_stream;
  h->ws = nullptr; h->ws_bytes = 0;
  h->tables_uploaded = false;
  h->have_forward = false;
  h->fwd_buf = 0;
  h->opt_graphs = 1;
  h->opt_kernel = 5;
  h->opt_tile_y = 8;
  h->opt_zchunk = 8;
  h->opt_zchunk_fwd = -1;
  h->opt_zchunk_fwd2 = -1;
  h->opt_zgroups = 0;
  h->zfork = nullptr;
  h->opt_sample = 0;
  h->opt_stages = 2;
  h->opt_pdl = 0;
  h->opt_prefetch = 0;
  h->opt_tile_x = 32;
  h->opt_compact = 1;
  h->opt_exact = 0;
  h->opt_inject_wait = 0;
  h->opt_reverse = 0;
  h->opt_forward = 0;
  for (int q = 0; q < FDTD_K_KINDS; ++q) {
    h->savg[q] = 0.f;
    h->scount[q] = 0;
  }
  h->cuda_ready = false;
  h->launches_fwd = h->launches_bwd = 0;
  h->fwd_ms = h->bwd_ms = 0.f;
  h->host_call_ms = 0.f;
  build_profiles(h);
  build_source(h);
  build_faces(h);
  *out = h;
  return FDTD_OK;
}

extern "C" const char* fdtd_last_error(const fdtd_handle* h) {
  return h ? h->err.c_str() : g_create_error.c_str();
}

static void drop_graphs(fdtd_handle* h) {
  for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second.exec);
  h->graphs.clear();
}

extern "C" int fdtd_destroy(fdtd_handle* h) {
  if (!h) return FDTD_OK;
  if (h->cuda_ready) {
    cudaStreamSynchronize(h->stream);
    drop_graphs(h);
    for (int d = 0; d < 2; ++d)
      for (int e = 0; e < 2; ++e)
        for (cudaEvent_t ev : h->spool[d][e]) cudaEventDestroy(ev);
    cudaEventDestroy(h->ev_in); cudaEventDestroy(h->ev_out);
    cudaEventDestroy(h->t0); cudaEventDestroy(h->t1);
    cudaEventDestroy(h->t2); cudaEventDestroy(h->t3);
    cudaEventDestroy(h->t4); cudaEventDestroy(h->t5);
    for (cudaEvent_t ev : h->zev) cudaEventDestroy(ev);
    for (cudaStream_t st : h->zs) cudaStreamDestroy(st);
    if (h->zfork) cudaEventDestroy(h->zfork);
    drop_batch(h);
    cudaStreamDestroy(h->stream);
  }
  delete h;
  return FDTD_OK;
}

extern "C" int fdtd_workspace_bytes(const fdtd_handle* h, const fdtd_record_cfg* rec,
                                    size_t* bytes) {
  if (!h || !bytes) return FDTD_EINVAL;
  if (rec && (rec->k < 1 || !valid_dtype(rec->dtype) || !coeffs_ok(rec))) return FDTD_EINVAL;
  *bytes = layout_of(h, rec).total;
  return FDTD_OK;
}

extern "C" int fdtd_tape_bytes(const fdtd_handle* h, const fdtd_record_cfg* rec, size_t* bytes) {
  if (!h || !bytes || !rec || rec->k < 1 || !valid_dtype(rec->dtype) || !coeffs_ok(rec))
    return FDTD_EINVAL;
  size_t J = n_samples(h->N, rec->k);
  size_t b;
  if (rec->dtype == kTapeBdct) {   // codes and per-block scales, unpadded
    const BdctLayout bl = bdct_layout(h->faces, bdct_coeffs(rec));
    b = J * (size_t)bl.bstart[6] * (bl.K + sizeof(float));
  } else {
    b = J * (size_t)sample_elems(h) * code_bytes(rec->dtype);
    if (rec->scaled) b += J * 6 * sizeof(float);
  }
  *bytes = b;
  return FDTD_OK;
}

extern "C" int fdtd_bind_workspace(fdtd_handle* h, void* dptr, size_t bytes) {
  if (!h) return FDTD_EINVAL;
  if (!dptr || ((uintptr_t)dptr & 255)) return fail(h, FDTD_EINVAL, "workspace must be 256-byte aligned");
  if (bytes < layout_of(h, nullptr).tape) return fail(h, FDTD_ENOMEM, "workspace too small");
  if (h->cuda_ready) cudaStreamSynchronize(h->stream);
  drop_graphs(h);
  h->ws = (char*)dptr;
  h->ws_bytes = bytes;
  h->tables_uploaded = false;
  h->have_forward = false;
  return FDTD_OK;
}

extern "C" int fdtd_set_option(fdtd_handle* h, int option, int value) {
  if (!h) return FDTD_EINVAL;
  switch (option) {
    case FDTD_OPT_USE_GRAPHS: h->opt_graphs = value ? 1 : 0; break;
    case FDTD_OPT_KERNEL:
      if (value != 0 && value != 5) return fail(h, FDTD_EINVAL, "kernel must be 0 or 5");
      if (value != h->opt_kernel) h->have_forward = false;   // the workspace layout changes
      h->opt_kernel = value;
      break;
    case FDTD_OPT_TILE_Y:
      if (value != 1 && value != 2 && value != 4 && value != 8 && value != 16)
        return fail(h, FDTD_EINVAL, "tile_y must be 1, 2, 4, 8 or 16");
      h->opt_tile_y = value;
      break;
    case FDTD_OPT_ZCHUNK:
      if (value < 0) return fail(h, FDTD_EINVAL, "zchunk must be >= 0");
      h->opt_zchunk = value;
      break;
    case FDTD_OPT_SAMPLE_EVERY:
      if (value < 0) return fail(h, FDTD_EINVAL, "sample interval must be >= 0");
      h->opt_sample = value;
      break;
    case FDTD_OPT_STAGES:
      if (value < 2 || value > 4) return fail(h, FDTD_EINVAL, "stages must be 2, 3 or 4");
      h->opt_stages = value;
      break;
    case FDTD_OPT_PDL: h->opt_pdl = value ? 1 : 0; break;
    case FDTD_OPT_PREFETCH: h->opt_prefetch = value ? 1 : 0; break;
    case FDTD_OPT_TILE_X:
      if (value != 32 && value != 40) return fail(h, FDTD_EINVAL, "tile_x must be 32 or 40");
      h->opt_tile_x = value;
      break;
    case FDTD_OPT_COMPACT_AUX:
      if ((value ? 1 : 0) != h->opt_compact) h->have_forward = false;   // layout changes
      h->opt_compact = value ? 1 : 0;
      break;
    case FDTD_OPT_ZCHUNK_FWD:
      if (value < -1) return fail(h, FDTD_EINVAL, "forward zchunk must be >= -1");
      h->opt_zchunk_fwd = value;
      break;
    case FDTD_OPT_ZCHUNK_FWD2:
      if (value < -1) return fail(h, FDTD_EINVAL, "two-step zchunk must be >= -1");
      h->opt_zchunk_fwd2 = value;
      break;
    case FDTD_OPT_ZGROUPS:
      if (value < 0 || value > kMaxZGroups) return fail(h, FDTD_EINVAL, "zgroups must be 0..16");
      h->opt_zgroups = value;
      break;
    case FDTD_OPT_REVERSE:
      if (value < 0 || value > 2) return fail(h, FDTD_EINVAL, "reverse must be 0, 1 or 2");
      if (value != h->opt_reverse) h->have_forward = false;   // the workspace layout changes
      h->opt_reverse = value;
      break;
    case FDTD_OPT_FORWARD:
      if (value < 0 || value > 3) return fail(h, FDTD_EINVAL, "forward must be 0, 1, 2 or 3");
      if (value != h->opt_forward) h->have_forward = false;   // the workspace layout changes
      h->opt_forward = value;
      break;
    case FDTD_OPT_INJECT_WAIT_TIMEOUT:
      if (value < 0) return fail(h, FDTD_EINVAL, "injected wait limit must be >= 0");
      h->opt_inject_wait = value;
      break;
    case FDTD_OPT_EXACT_REVERSAL:
      if (value != 0 && (value < 8 || value > 30))
        return fail(h, FDTD_EINVAL, "exact reversal: q must be 0 or 8..30");
      if (value != h->opt_exact) h->have_forward = false;   // the backward must match it
      h->opt_exact = value;
      break;
    default: return fail(h, FDTD_EINVAL, "unknown option");
  }
  return FDTD_OK;
}

extern "C" int fdtd_get_option(const fdtd_handle* h, int option, int* value) {
  if (!h || !value) return FDTD_EINVAL;
  switch (option) {
    case FDTD_OPT_USE_GRAPHS: *value = h->opt_graphs; break;
    case FDTD_OPT_KERNEL: *value = h->opt_kernel; break;
    case FDTD_OPT_TILE_Y: *value = h->opt_tile_y; break;
    case FDTD_OPT_ZCHUNK: *value = h->opt_zchunk; break;
    case FDTD_OPT_SAMPLE_EVERY: *value = h->opt_sample; break;
    case FDTD_OPT_STAGES: *value = h->opt_stages; break;
    case FDTD_OPT_PDL: *value = h->opt_pdl; break;
    case FDTD_OPT_PREFETCH: *value = h->opt_prefetch; break;
    case FDTD_OPT_TILE_X: *value = h->opt_tile_x; break;
    case FDTD_OPT_COMPACT_AUX: *value = h->opt_compact; break;
    case FDTD_OPT_EXACT_REVERSAL: *value = h->opt_exact; break;
    case FDTD_OPT_ZCHUNK_FWD: *value = h->opt_zchunk_fwd; break;
    case FDTD_OPT_ZCHUNK_FWD2: *value = h->opt_zchunk_fwd2; break;
    case FDTD_OPT_ZGROUPS: *value = h->opt_zgroups; break;
    case FDTD_OPT_INJECT_WAIT_TIMEOUT: *value = h->opt_inject_wait; break;
    case FDTD_OPT_REVERSE: *value = h->opt_reverse; break;
    case FDTD_OPT_FORWARD: *value = h->opt_forward; break;
    default: return FDTD_EINVAL;
  }
  return FDTD_OK;
}

// ------------------------------------------------------ introspection ---
extern "C" int fdtd_pml_profile(const fdtd_handle* h, int axis, int which, float* out) {
  if (!h || !out || axis < 0 || axis > 2 || which < 0 || which > 5) return FDTD_EINVAL;
  int n = axis == 0 ? h->nx : (axis == 1 ? h->ny : h->nz);
  memcpy(out, &h->prof[(axis * 6 + which) * h->nmax], n * sizeof(float));
  return FDTD_OK;
}

extern "C" int fdtd_source_waveform(const fdtd_handle* h, float* out) {
  if (!h || !out) return FDTD_EINVAL;
  memcpy(out, h->wave.data(), h->N * sizeof(float));
  return FDTD_OK;
}

extern "C" int fdtd_interp_weights(const fdtd_handle* h, const fdtd_record_cfg* rec, int step,
                                   int field, int* slot, float* weight) {
  if (!h || !rec || !slot || !weight || rec->k < 1 || step < 0 || step >= h->N ||
      (field != 0 && field != 1))
    return FDTD_EINVAL;
  interp_weights(h, rec, step, field, slot, weight);
  return FDTD_OK;
}

// --------------------------------------------------------- orchestration ---
static int ensure_cuda(fdtd_handle* h) {
  if (h->cuda_ready) return FDTD_OK;
  CK(h, cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
  CK(h, cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming));
  CK(h, cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming));
  CK(h, cudaEventCreate(&h->t0));
  CK(h, cudaEventCreate(&h->t1));
  CK(h, cudaEventCreate(&h->t2));
  CK(h, cudaEventCreate(&h->t3));
  CK(h, cudaEventCreate(&h->t4));
  CK(h, cudaEventCreate(&h->t5));
  h->cuda_ready = true;
  return FDTD_OK;
}

static int begin(fdtd_handle* h) {
  if (!h->ws) return fail(h, FDTD_ESTATE, "no workspace bound");
  int rc = ensure_cuda(h);
  if (rc) return rc;
  CK(h, cudaEventRecord(h->ev_in, h->user_stream));
  CK(h, cudaStreamWaitEvent(h->stream, h->ev_in, 0));
  if (!h->tables_uploaded) {
    Layout L = layout_of(h, nullptr);
    CK(h, cudaMemcpyAsync(h->ws + L.prof, h->prof.data(), h->prof.size() * sizeof(float),
                          cudaMemcpyHostToDevice, h->stream));
    if (!h->srcw.empty())
      CK(h, cudaMemcpyAsync(h->ws + L.srcw, h->srcw.data(), h->srcw.size() * sizeof(float),
                            cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));  // host vectors may be pageable
    h->tables_uploaded = true;
  }
  return FDTD_OK;
}

static int finish(fdtd_handle* h) {
  CK(h, cudaEventRecord(h->ev_out, h->stream));
  CK(h, cudaStreamWaitEvent(h->user_stream, h->ev_out, 0));
  return FDTD_OK;
}

// Tile height the staged kernels run with: they cover two tile rows per
// warp, so their tiles are at least 2 high.
static int lag_tile_y(const fdtd_handle* h) {
  return (h->opt_kernel == 5 && h->opt_tile_y < 2) ? 2 : h->opt_tile_y;
}

// Tile width of the two-cells-per-thread kernels: 40-wide tiles exist for a
// tile height of 8 with 2 or 3 stages, otherwise 32.
static int lag_tile_x(const fdtd_handle* h) {
  if (h->opt_kernel != 5 || lag_tile_y(h) != 8 || h->opt_stages > 3) return 32;
  return h->opt_tile_x == 40 ? 40 : 32;
}

static Det det_of(const fdtd_detector& d) {
  Det o;
  o.kind = d.kind;
  o.axis = d.axis;
  o.index = d.index;
  o.u0 = d.lo[0]; o.u1 = d.hi[0];
  o.v0 = d.lo[1]; o.v1 = d.hi[1];
  return o;
}

static Det det2_of(const fdtd_handle* h) { return det_of(h->det2); }

// z groups of kernel 5's half-steps in direction dir (0 forward, 1 reverse).
// Automatic (0): 4 in the forward and 3 in the reverse, the fastest counts on
// both 200 x 200 x 100 and 600 x 600 x 300 (the reverse phases join at every
// step's restore, so only two phases overlap there).
static int zgroups_of(const fdtd_handle* h, int dir) {
  if (h->opt_kernel != 5) return 1;
  if (h->opt_zgroups > 0) return h->opt_zgroups;
  return dir == 0 ? 4 : 3;
}

// z chunk of kernel 5's forward half-steps.  Automatic (-1): with z groups
// the reverse phases' chunk (8 planes by default: 7 % faster than one launch
// per half-step on 200 x 200 x 100); without, 16 planes when the 16-plane
// grid of CTAs fits in about one wave of resident CTAs (8 per SM for these
// kernels), else the reverse phases' chunk: on small grids the longer chunks
// halve the halo planes and the ramps without adding a second wave
// (measured: 3 % faster forward on 200 x 200 x 100, 1 % slower on
// 600 x 600 x 300 where the rule keeps 8).
static int forward_zchunk(const fdtd_handle* h, const StepArgs& a) {
  if (h->opt_zchunk_fwd == 0) return h->nz;
  if (h->opt_zchunk_fwd > 0) return h->opt_zchunk_fwd;
  if (zgroups_of(h, 0) > 1) return a.zchunk;
  static int sms = 0;
  if (!sms) {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
      sms = n;
  }
  const long long tiles = (long long)((h->nx + a.tile_x - 1) / a.tile_x) *
                          ((h->ny + a.tile_y - 1) / a.tile_y);
  const long long units16 = tiles * ((h->nz + 15) / 16);
  return sms > 0 && units16 * 20 <= 8LL * sms * 21 ? 16 : a.zchunk;
}

static StepArgs step_args(const fdtd_handle* h, const Layout& L) {
  StepArgs a;
  memset(&a, 0, sizeof a);
  a.g = geo_of(h);
  a.g.prof = (const float*)(h->ws + L.prof);
  a.cb = (float*)(h->ws + L.cb);
  a.gacc = (double*)(h->ws + L.gacc);
  for (int i = 0; i < 3; ++i) { a.dlo[i] = h->dlo[i]; a.dhi[i] = h->dhi[i]; }
  a.src.kind = h->src.kind;
  a.src.comp = h->src.component;
  a.src.axis = h->src_axis;
  a.src.index = h->src_index;
  a.src.u0 = h->src_u0; a.src.u1 = h->src_u1; a.src.v0 = h->src_v0; a.src.v1 = h->src_v1;
  a.src.w = (const float*)(h->ws + L.srcw);
  a.det = det_of(h->det);
  a.tile_y = lag_tile_y(h);
  a.stages = h->opt_stages;
  a.pdl = h->opt_pdl;
  a.prefetch = h->opt_prefetch;
  a.tile_x = lag_tile_x(h);
  a.xq = h->opt_exact;
  a.xs = h->opt_exact ? ldexpf(1.0f, h->opt_exact) : 1.0f;
  a.xi = h->opt_exact ? ldexpf(1.0f, -h->opt_exact) : 1.0f;
  a.zchunk = h->opt_zchunk > 0 ? h->opt_zchunk : h->nz;
  a.err = (unsigned*)(h->ws + L.err);
  return a;
}

// Sampled kernel timing: event pairs recorded on h->stream around every
// opt_sample-th launch of a kernel kind (external event nodes when captured).
// Sampled kernel timing.  A CUDA event pair around a single launch inside the
// time loop also measures the event nodes and the launch latency they expose
// (several microseconds), so the per-launch cost is measured differentially:
// every m-th launch opens an interval, alternately around one launch (kind p)
// and around two consecutive launches (kind p, then kind q).  The in-loop
// cost of kind q is mean(pair p->q) - mean(single p): both intervals carry the
// same event overhead, which cancels, and what remains is q's duration plus
// its launch gap after p, i.e. what q adds to the loop.
struct Sampler {
  fdtd_handle* h;
  int dir;
  long long m, i = 0;
  int open = -1;        // plan entry of the open interval
  int open_type = 0;
  long long end_at = 0;  // launch index after which it closes
  Sampler(fdtd_handle* h_, int dir_) : h(h_), dir(dir_), m(h_->opt_sample) {
    h->splan[dir].clear();
  }
  cudaError_t record(int which, size_t slot) {
    std::vector<cudaEvent_t>& pool = h->spool[dir][which];
    while (pool.size() <= slot) {
      cudaEvent_t ev;
      cudaError_t e = cudaEventCreate(&ev);
      if (e) return e;
      pool.push_back(ev);
    }
    return cudaEventRecordWithFlags(pool[slot], h->stream, cudaEventRecordExternal);
  }
  // A fixed integer hash of the launch index picks the sampled launches (one
  // in m on average) and the interval type, so that every kind is sampled
  // both alone and after each of its predecessors whatever the number of
  // launches per time step (a plain every-m-th choice with alternating types
  // misses kinds when m shares a factor with it).
  static uint32_t mix(uint64_t v) {
    v ^= v >> 33;
    v *= 0xff51afd7ed558ccdULL;
    v ^= v >> 33;
    v *= 0xc4ceb9fe1a85ec53ULL;
    v ^= v >> 33;
    return (uint32_t)v;
  }
  cudaError_t before(int kind) {
    if (m <= 0 || open >= 0) return cudaSuccess;
    const uint32_t hsh = mix((uint64_t)i);
    if (hsh % (uint32_t)m) return cudaSuccess;
    // no interval beyond the events created before the capture
    if (h->splan[dir].size() >= h->spool[dir][0].size() ||
        h->splan[dir].size() >= h->spool[dir][1].size())
      return cudaSuccess;
    open_type = (int)((hsh >> 24) & 1);
    h->splan[dir].push_back(SampleEntry{-1, kind, kind});
    open = (int)h->splan[dir].size() - 1;
    end_at = i + open_type;
    return record(0, (size_t)open);
  }
  cudaError_t after(int kind) {
    cudaError_t e = cudaSuccess;
    if (open >= 0 && i == end_at) {
      SampleEntry& se = h->splan[dir][open];
      se.type = open_type;
      se.q = kind;
      e = record(1, (size_t)open);
      open = -1;
    }
    ++i;
    return e;
  }
};

static void collect_samples(fdtd_handle* h, int dir, const int* kinds, int nk) {
  const std::vector<SampleEntry>& plan = h->splan[dir];
  double ssum[FDTD_K_KINDS] = {0}, psum[FDTD_K_KINDS][FDTD_K_KINDS] = {{0}};
  int sn[FDTD_K_KINDS] = {0}, pn[FDTD_K_KINDS][FDTD_K_KINDS] = {{0}};
  for (size_t j = 0; j < plan.size(); ++j) {
    const SampleEntry& se = plan[j];
    if (se.type < 0) continue;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->spool[dir][0][j], h->spool[dir][1][j]) != cudaSuccess) continue;
    if (se.type == 0) {
      ssum[se.p] += ms;
      ++sn[se.p];
    } else {
      psum[se.p][se.q] += ms;
      ++pn[se.p][se.q];
    }
  }
  for (int t = 0; t < nk; ++t) {
    const int q = kinds[t];
    int best = -1;
    for (int p = 0; p < FDTD_K_KINDS; ++p)
      if (pn[p][q] > 0 && sn[p] > 0 && (best < 0 || pn[p][q] > pn[best][q])) best = p;
    if (best >= 0) {
      h->savg[q] = (float)(psum[best][q] / pn[best][q] - ssum[best] / sn[best]);
      h->scount[q] = std::min(pn[best][q], sn[best]);
    } else {
      h->savg[q] = 0.f;
      h->scount[q] = 0;
    }
  }
}

// Chunks [lo, hi) of group g when nch z chunks are split into G <= nch groups
// (every range non-empty).
static void zgroup_range(int nch, int G, int g, int* lo, int* hi) {
  *lo = (int)((long long)g * nch / G);
  *hi = (int)((long long)(g + 1) * nch / G);
}

// z-group scheduling of the two-cells-per-thread half-steps (FDTD_OPT_ZGROUPS):
// each half-step launch is split into G launches over consecutive ranges of its
// z chunks, group g on its own stream.  A half-step reads what the previous one
// wrote at most one plane beyond its own cells, and a chunk range spans at least
// one plane, so group g of a phase waits only for groups g - 1 and g + 1 of the
// phase before (and for its own through stream order); the tail of one phase
// then overlaps the start of the next.  Launches that read or write whole faces
// (tape record and restore, the second detector's monitor) run on the main
// stream between a join of all groups and a fork.
struct ZGroups {
  fdtd_handle* h;
  int G = 1, nch = 1, par = 0;
  bool forked = false, prev = false;
  ZGroups(fdtd_handle* h_, bool on, int dir, const StepArgs& a) : h(h_) {
    nch = (a.g.nz + a.zchunk - 1) / a.zchunk;
    const int want = zgroups_of(h, dir);
    if (on && want > 1 && h->zfork && (int)h->zs.size() >= want &&
        h->zev.size() >= 3 * h->zs.size())
      G = std::min(want, nch);
  }
  bool active() const { return G > 1; }
  cudaEvent_t ev(int slot, int g) const { return h->zev[(size_t)g * 3 + slot]; }
  cudaError_t fork() {
    if (!active()) return cudaSuccess;
    cudaError_t e = cudaEventRecord(h->zfork, h->stream);
    for (int g = 0; !e && g < G; ++g) e = cudaStreamWaitEvent(h->zs[g], h->zfork, 0);
    forked = true;
    prev = false;
    return e;
  }
  cudaError_t join() {
    if (!active() || !forked) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    for (int g = 0; !e && g < G; ++g) {
      e = cudaEventRecord(ev(2, g), h->zs[g]);
      if (!e) e = cudaStreamWaitEvent(h->stream, ev(2, g), 0);
    }
    forked = false;
    return e;
  }
  template <class Launch>
  cudaError_t phase(Launch launch, StepArgs a) {
    cudaError_t e = cudaSuccess;
    for (int g = 0; g < G; ++g) {
      cudaStream_t st = h->zs[g];
      if (prev && g > 0 && (e = cudaStreamWaitEvent(st, ev(par ^ 1, g - 1), 0))) return e;
      if (prev && g + 1 < G && (e = cudaStreamWaitEvent(st, ev(par ^ 1, g + 1), 0))) return e;
      zgroup_range(nch, G, g, &a.zc0, &a.zc1);
      if ((e = launch(a, st))) return e;
      if ((e = cudaEventRecord(ev(par, g), st))) return e;
    }
    par ^= 1;
    prev = true;
    return e;
  }
};

// Streams and events of the z-group scheduling of direction dir (created as
// needed, outside a capture).
static cudaError_t ensure_zgroups(fdtd_handle* h, int dir) {
  const int want = zgroups_of(h, dir);
  if (want <= 1 || (int)h->zs.size() >= want) return cudaSuccess;
  cudaError_t e = cudaSuccess;
  if (!h->zfork) e = cudaEventCreateWithFlags(&h->zfork, cudaEventDisableTiming);
  while (!e && (int)h->zs.size() < want) {
    // a stream joins the pool only with its three events
    cudaStream_t st;
    cudaEvent_t evs[3] = {nullptr, nullptr, nullptr};
    e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e) break;
    for (int i = 0; !e && i < 3; ++i) e = cudaEventCreateWithFlags(&evs[i], cudaEventDisableTiming);
    if (e) {
      for (cudaEvent_t ev : evs)
        if (ev) cudaEventDestroy(ev);
      cudaStreamDestroy(st);
      break;
    }
    h->zs.push_back(st);
    h->zev.insert(h->zev.end(), evs, evs + 3);
  }
  return e;
}

static const int kFwdKinds[] = {FDTD_K_FWD_H, FDTD_K_FWD_E, FDTD_K_RECORD, FDTD_K_MONITOR,
                                FDTD_K_FWD_FUSED, FDTD_K_FWD_2STEP};
static const int kBwdKinds[] = {FDTD_K_RESTORE, FDTD_K_REV_E, FDTD_K_REV_H, FDTD_K_REV_PRIMAL,
                                FDTD_K_REV_ADJOINT, FDTD_K_REV_ADJOINT_CPML};

// Enqueue the forward time loop on h->stream (capturable).
static cudaError_t enqueue_forward(fdtd_handle* h, const fdtd_record_cfg* rec, int* launches) {
  Layout L = layout_of(h, rec);
  StepArgs a = step_args(h, L);
  a.pl = L.plF;
  if (h->opt_kernel == 5) a.zchunk = forward_zchunk(h, a);
  size_t nc6 = 6 * (size_t)a.g.nc * sizeof(float);
  size_t psb = (size_t)L.plF.total * sizeof(float);
  cudaError_t e;
  int nl = 0;
  if ((e = cudaMemsetAsync(h->ws + L.F[0], 0, nc6, h->stream))) return e;
  if ((e = cudaMemsetAsync(h->ws + L.psiF[0], 0, psb, h->stream))) return e;
  if ((e = cudaMemsetAsync(h->ws + L.obj, 0, h->N * sizeof(double), h->stream))) return e;
  int r = (h->N - 1) % rec->k;
  const bool pair = h->opt_kernel == 5;
  LagMaps lmaps;
  if (pair &&
      (e = encode_lag_maps((const float*)(h->ws + L.F[0]), (const float*)(h->ws + L.F[0]),
                           (const float*)(h->ws + L.cb), (const float*)(h->ws + L.psiF[0]), a.g,
                           a.tile_y, a.tile_x, L.plF, &lmaps)))
    return e;
  a.F = (float*)(h->ws + L.F[0]);
  a.psiA = (float*)(h->ws + L.psiF[0]);
  char* tape = h->ws + L.tape;
  float* scales = (float*)(h->ws + L.scales);
  const bool bdct = rec->dtype == kTapeBdct;
  const int eb = bdct ? 1 : code_bytes(rec->dtype);
  const BdctLayout bl = bdct ? bdct_layout(h->faces, bdct_coeffs(rec)) : BdctLayout{};
  auto record = [&](const float* FH, const float* FE, int j) {
    void* smp = tape + (size_t)j * L.stride * eb;
    return bdct ? launch_record_bdct(FH, FE, a.g, h->faces, bl, smp, h->stream)
                : launch_record(rec->dtype, rec->scaled, FH, FE, a.g, h->faces, smp,
                                scales + (size_t)j * 6, h->stream);
  };
  const Det det2 = det2_of(h);
  if (det2.kind && (e = cudaMemsetAsync(h->ws + L.obj2, 0, h->N * sizeof(double), h->stream)))
    return e;
  Sampler smp(h, 0);
  if (two_step_forward(h)) {
    // two steps per pass: steps n, n + 1 of the deep units in one launch on
    // the main stream (buffer cur -> cur ^ 1, the intermediate level's frame
    // -> buffer 2), the split H half-step of step n over the other units
    // beside it on a side stream (cur -> 2), then their split E half-step of
    // step n (cur -> 2) and both half-steps of step n + 1 (2 -> cur ^ 1); the
    // auxiliaries stay in place.  An odd count runs step 0 as split
    // half-steps over every unit (cur -> cur ^ 1).
    const int zcs = fused_forward_zchunk(h);
    a.zchunk = zcs;
    const RevUnits D = deep_units(a.g, zcs);
    RevUnits all = D;   // no deep box: the ring decode covers every unit
    all.ix0 = all.ix1 = all.iy0 = all.iy1 = all.iz0 = all.iz1 = 0;
    // planes per CTA of the pass: 16 split chunks by default (600 x 600 x 300,
    // 1000-step runs: 1055, 1036 and 1028 us per forward step with 4, 8 and
    // 16 chunks; each chunk re-reads two planes below and one above it)
    const int zdeep = h->opt_zchunk_fwd2 > 0 ? h->opt_zchunk_fwd2 : 16 * zcs;
    const float* Fb[3];
    for (int b = 0; b < 3; ++b) Fb[b] = (const float*)(h->ws + L.F[b]);
    const float* cbp = (const float*)(h->ws + L.cb);
    const float* ps = (const float*)(h->ws + L.psiF[0]);
    Fwd2Maps dm[2];
    LagMaps lh[3], le[3][3];   // le[i][o]: E of buffer i, Ht^{n+1/2} of buffer o
    for (int b = 0; b < 3; ++b) {
      if (b < 2 && (e = encode_fwd2_maps(Fb[b], cbp, a.g, &dm[b]))) return e;
      if ((e = encode_lag_maps(Fb[b], Fb[b], cbp, ps, a.g, 8, 32, L.plF, &lh[b]))) return e;
      for (int o = 0; o < 3; ++o)
        if (o != b && (e = encode_lag_maps(Fb[b], Fb[b], cbp, ps, a.g, 8, 32, L.plF, &le[b][o],
                                           Fb[o])))
          return e;
    }
    const bool conc = h->opt_sample == 0 && h->opt_zgroups != 1 && !h->zs.empty() &&
                      h->zev.size() >= 3;
    // one split time step over the units of U (umode 1 and 2) from buffer i
    // into buffer o, with its record and second detector
    auto split_step = [&](int n, int i, int o, const RevUnits& U, cudaStream_t hs,
                          bool h_done) -> cudaError_t {
      StepArgs b = a;
      b.U = U;
      b.zchunk = zcs;
      b.jn = h->wave[n];
      b.obj = (double*)(h->ws + L.obj) + n;
      b.F = (float*)(h->ws + L.F[i]);
      b.Fn = (float*)(h->ws + L.F[o]);
      cudaError_t e2;
      if (!h_done) {
        if ((e2 = smp.before(FDTD_K_FWD_H))) return e2;
        for (int um = 1; um <= 2; ++um) {
          b.umode = um;
          if ((e2 = launch_lag2(0, lh[i], b, hs))) return e2;
        }
        if ((e2 = smp.after(FDTD_K_FWD_H))) return e2;
        nl += 2;
        return cudaSuccess;
      }
      if ((e2 = smp.before(FDTD_K_FWD_E))) return e2;
      for (int um = 1; um <= 2; ++um) {
        b.umode = um;
        if ((e2 = launch_lag2(1, le[i][o], b, h->stream))) return e2;
      }
      if ((e2 = smp.after(FDTD_K_FWD_E))) return e2;
      nl += 2;
      const bool rec_now = n >= r && (n - r) % rec->k == 0;
      if (rec_now) {   // E^n in buffer i, Ht^{n+1/2} in buffer o
        if ((e2 = smp.before(FDTD_K_RECORD))) return e2;
        if ((e2 = record(b.Fn, b.F, (n - r) / rec->k))) return e2;
        if ((e2 = smp.after(FDTD_K_RECORD))) return e2;
        ++nl;
      }
      if (det2.kind) {
        if ((e2 = smp.before(FDTD_K_MONITOR))) return e2;
        if ((e2 = launch_monitor(b.Fn, a.g, det2, (double*)(h->ws + L.obj2) + n, h->stream)))
          return e2;
        if ((e2 = smp.after(FDTD_K_MONITOR))) return e2;
        ++nl;
      }
      return cudaSuccess;
    };
    int cur = 0, n = 0;
    if (h->N & 1) {
      if ((e = split_step(0, cur, cur ^ 1, all, h->stream, false))) return e;
      if ((e = split_step(0, cur, cur ^ 1, all, h->stream, true))) return e;
      cur ^= 1;
      n = 1;
    }
    for (; n + 1 < h->N; n += 2) {
      cudaStream_t side = conc ? h->zs[0] : h->stream;
      if (conc) {
        if ((e = cudaEventRecord(h->zev[0], h->stream))) return e;
        if ((e = cudaStreamWaitEvent(side, h->zev[0], 0))) return e;
      }
      StepArgs b = a;
      b.F = (float*)(h->ws + L.F[cur]);
      b.Fn = (float*)(h->ws + L.F[cur ^ 1]);
      b.Fm = (float*)(h->ws + L.F[2]);
      b.zcs = zcs;
      b.zchunk = zdeep;
      if ((e = smp.before(FDTD_K_FWD_2STEP))) return e;
      if ((e = launch_fwd_2step(dm[cur], b, D, h->stream))) return e;
      if ((e = smp.after(FDTD_K_FWD_2STEP))) return e;
      ++nl;
      if ((e = split_step(n, cur, 2, D, side, false))) return e;
      if (conc) {
        if ((e = cudaEventRecord(h->zev[1], side))) return e;
        if ((e = cudaStreamWaitEvent(h->stream, h->zev[1], 0))) return e;
      }
      if ((e = split_step(n, cur, 2, D, h->stream, true))) return e;
      if ((e = split_step(n + 1, 2, cur ^ 1, D, h->stream, false))) return e;
      if ((e = split_step(n + 1, 2, cur ^ 1, D, h->stream, true))) return e;
      cur ^= 1;
    }
    *launches = nl;
    return cudaSuccess;
  }
  if (fused_forward(h)) {
    // fused forward step: the CPML-free units in one launch on the main
    // stream, the split H half-step of the other units beside it on a side
    // stream, then their split E half-step; buffer cur of the fields is read
    // and buffer cur ^ 1 written (the auxiliaries stay in place)
    a.zchunk = fused_forward_zchunk(h);
    const RevUnits U = rev_units(a.g, a.zchunk);
    RevMaps fm[2];
    LagMaps lh[2], le[2];
    for (int b = 0; b < 2; ++b) {
      const float* Fb = (const float*)(h->ws + L.F[b]);
      const float* Fo = (const float*)(h->ws + L.F[b ^ 1]);
      const float* cbp = (const float*)(h->ws + L.cb);
      const float* ps = (const float*)(h->ws + L.psiF[0]);
      if ((e = encode_rev_maps(Fb, Fb, cbp, ps, a.g, L.plF, &fm[b]))) return e;
      if ((e = encode_lag_maps(Fb, Fb, cbp, ps, a.g, 8, 32, L.plF, &lh[b]))) return e;
      if ((e = encode_lag_maps(Fb, Fb, cbp, ps, a.g, 8, 32, L.plF, &le[b], Fo))) return e;
    }
    const bool conc = h->opt_sample == 0 && h->opt_zgroups != 1 && !h->zs.empty() &&
                      h->zev.size() >= 3;
    int cur = 0;
    for (int n = 0; n < h->N; ++n) {
      a.jn = h->wave[n];
      a.obj = (double*)(h->ws + L.obj) + n;
      a.F = (float*)(h->ws + L.F[cur]);
      a.Fn = (float*)(h->ws + L.F[cur ^ 1]);
      const bool rec_now = n >= r && (n - r) % rec->k == 0;
      const int j = rec_now ? (n - r) / rec->k : 0;
      cudaStream_t side = conc ? h->zs[0] : h->stream;
      if (conc) {
        if ((e = cudaEventRecord(h->zev[0], h->stream))) return e;
        if ((e = cudaStreamWaitEvent(side, h->zev[0], 0))) return e;
      }
      StepArgs b = a;
      b.U = U;
      if ((e = smp.before(FDTD_K_FWD_FUSED))) return e;
      if ((e = launch_fwd_fused(fm[cur], a, U, h->stream))) return e;
      if ((e = smp.after(FDTD_K_FWD_FUSED))) return e;
      if ((e = smp.before(FDTD_K_FWD_H))) return e;
      for (int um = 1; um <= 2; ++um) {
        b.umode = um;
        if ((e = launch_lag2(0, lh[cur], b, side))) return e;
      }
      if ((e = smp.after(FDTD_K_FWD_H))) return e;
      if (conc) {
        if ((e = cudaEventRecord(h->zev[1], side))) return e;
        if ((e = cudaStreamWaitEvent(h->stream, h->zev[1], 0))) return e;
      }
      if ((e = smp.before(FDTD_K_FWD_E))) return e;
      for (int um = 1; um <= 2; ++um) {
        b.umode = um;
        if ((e = launch_lag2(1, le[cur], b, h->stream))) return e;
      }
      if ((e = smp.after(FDTD_K_FWD_E))) return e;
      nl += 5;
      if (rec_now) {   // E^n is still in buffer cur, Ht^{n+1/2} now in cur ^ 1
        if ((e = smp.before(FDTD_K_RECORD))) return e;
        if ((e = record(a.Fn, a.F, j))) return e;
        if ((e = smp.after(FDTD_K_RECORD))) return e;
        ++nl;
      }
      if (det2.kind) {
        if ((e = smp.before(FDTD_K_MONITOR))) return e;
        if ((e = launch_monitor(a.Fn, a.g, det2, (double*)(h->ws + L.obj2) + n, h->stream)))
          return e;
        if ((e = smp.after(FDTD_K_MONITOR))) return e;
        ++nl;
      }
      cur ^= 1;
    }
    *launches = nl;
    return cudaSuccess;
  }
  ZGroups zg(h, pair, 0, a);
  if (zg.active()) smp.m = 0;   // launches of a phase overlap: no per-kind intervals
  if ((e = zg.fork())) return e;
  for (int n = 0; n < h->N; ++n) {
    a.jn = h->wave[n];
    a.obj = (double*)(h->ws + L.obj) + n;
    const bool rec_now = n >= r && (n - r) % rec->k == 0;
    const int j = rec_now ? (n - r) / rec->k : 0;
    if ((e = smp.before(FDTD_K_FWD_H))) return e;
    if (zg.active()) {
      if ((e = zg.phase([&](const StepArgs& b, cudaStream_t st) {
             return launch_lag2(0, lmaps, b, st); }, a)))
        return e;
      nl += zg.G - 1;
    } else if ((e = pair ? launch_lag2(0, lmaps, a, h->stream) : launch_fwd_h(a, h->stream))) {
      return e;
    }
    if ((e = smp.after(FDTD_K_FWD_H))) return e;
    ++nl;
    if (rec_now) {
      if ((e = zg.join())) return e;
      if ((e = smp.before(FDTD_K_RECORD))) return e;
      if ((e = record(a.F, a.F, j))) return e;
      if ((e = smp.after(FDTD_K_RECORD))) return e;
      if ((e = zg.fork())) return e;
      ++nl;
    }
    if ((e = smp.before(FDTD_K_FWD_E))) return e;
    if (zg.active()) {
      if ((e = zg.phase([&](const StepArgs& b, cudaStream_t st) {
             return launch_lag2(1, lmaps, b, st); }, a)))
        return e;
      nl += zg.G - 1;
    } else if ((e = pair ? launch_lag2(1, lmaps, a, h->stream) : launch_fwd_e(a, h->stream))) {
      return e;
    }
    if ((e = smp.after(FDTD_K_FWD_E))) return e;
    ++nl;
    if (det2.kind) {
      if ((e = zg.join())) return e;
      if ((e = smp.before(FDTD_K_MONITOR))) return e;
      if ((e = launch_monitor(a.F, a.g, det2, (double*)(h->ws + L.obj2) + n, h->stream))) return e;
      if ((e = smp.after(FDTD_K_MONITOR))) return e;
      if ((e = zg.fork())) return e;
      ++nl;
    }
  }
  if ((e = zg.join())) return e;
  *launches = nl;
  return cudaSuccess;
}

static cudaError_t enqueue_backward(fdtd_handle* h, const fdtd_record_cfg* rec, int* launches) {
  Layout L = layout_of(h, rec);
  StepArgs a = step_args(h, L);
  a.pl = L.plL;
  size_t nc6 = 6 * (size_t)a.g.nc * sizeof(float);
  size_t psb = (size_t)L.plL.total * sizeof(float);
  size_t nd = (size_t)(h->dhi[0] - h->dlo[0]) * (h->dhi[1] - h->dlo[1]) * (h->dhi[2] - h->dlo[2]);
  cudaError_t e;
  int nl = 0;
  // the adjoint starts at zero in the buffer the first step reads: the fused
  // reverse step starts in the forward's buffer, the split phases work in 0
  const int lam0 = fused_reverse(h) ? h->fwd_buf : 0;
  if ((e = cudaMemsetAsync(h->ws + L.L[lam0], 0, nc6, h->stream))) return e;
  if ((e = cudaMemsetAsync(h->ws + L.psiL[0], 0, psb, h->stream))) return e;
  if ((e = cudaMemsetAsync(h->ws + L.psiL[1], 0, psb, h->stream))) return e;
  if ((e = cudaMemsetAsync(h->ws + L.gacc, 0, nd * sizeof(double), h->stream))) return e;
  // failure-detection test hook: one bounded device wait that nothing
  // completes gives up after the set limit and sets the timeout bit
  if (h->opt_inject_wait > 0 &&
      (e = launch_wait_selftest(h->opt_inject_wait, (unsigned*)(h->ws + L.err), h->stream)))
    return e;
  a.F = (float*)(h->ws + L.F[h->fwd_buf]);
  a.L = (float*)(h->ws + L.L[0]);
  Det det = a.det;
  const Det det2 = det2_of(h);
  int cur = h->fwd_buf;   // the forward's final state
  const bool fused = fused_reverse(h);
  const bool rpair = h->opt_kernel == 5 && !fused;
  LagMaps lrmaps[2];
  for (int b = 0; b < 2; ++b)
    if (rpair && (e = encode_lag_maps(a.F, a.L, (const float*)(h->ws + L.cb),
                                      (const float*)(h->ws + L.psiL[b]), a.g, a.tile_y, a.tile_x,
                                      L.plL, &lrmaps[b])))
      return e;
  // fused reverse step: buffer cur of the fields, the adjoint fields and the
  // auxiliaries is read, buffer cur ^ 1 written (the forward's state is in
  // buffer fwd_buf; the adjoint starts in buffer fwd_buf too)
  RevMaps rmaps[2];
  const RevUnits U = rev_units(a.g, a.zchunk);
  // the adjoint launches run on a side stream unless kernel timing is being
  // sampled or one launch per half-step is asked for (FDTD_OPT_ZGROUPS = 1)
  const bool conc = fused && h->opt_sample == 0 && h->opt_zgroups != 1 && !h->zs.empty() &&
                    h->zev.size() >= 3;
  for (int b = 0; fused && b < 2; ++b)
    if ((e = encode_rev_maps((const float*)(h->ws + L.F[b]), (const float*)(h->ws + L.L[b]),
                             (const float*)(h->ws + L.cb), (const float*)(h->ws + L.psiL[b]), a.g,
                             L.plL, &rmaps[b])))
      return e;
  const BdctLayout bl =
      rec->dtype == kTapeBdct ? bdct_layout(h->faces, bdct_coeffs(rec)) : BdctLayout{};
  Sampler smp(h, 1);
  ZGroups zg(h, rpair, 1, a);
  if (zg.active()) smp.m = 0;   // launches of a phase overlap: no per-kind intervals
  for (int n = h->N - 1; n >= 0; --n) {
    if ((e = zg.join())) return e;
    if (fused) {
      a.F = (float*)(h->ws + L.F[cur]);
      a.L = (float*)(h->ws + L.L[cur]);
      a.Fn = (float*)(h->ws + L.F[cur ^ 1]);
      a.Ln = (float*)(h->ws + L.L[cur ^ 1]);
    }
    Interp ip;
    interp_weights(h, rec, n, 0, ip.slot[0], ip.w[0]);
    interp_weights(h, rec, n, 1, ip.slot[1], ip.w[1]);
    if ((e = smp.before(FDTD_K_RESTORE))) return e;
    if ((e = rec->dtype == kTapeBdct
                 ? launch_restore_seed_bdct(a.F, a.L, a.g, h->faces, bl, h->ws + L.tape, L.stride,
                                            ip, det, det2, (const double*)(h->ws + L.seeds),
                                            h->stream)
                 : launch_restore_seed(rec->dtype, a.F, a.L, a.g, h->faces, h->ws + L.tape,
                                       L.stride, (const float*)(h->ws + L.scales), ip, det, det2,
                                       (const double*)(h->ws + L.seeds), h->stream)))
      return e;
    if ((e = smp.after(FDTD_K_RESTORE))) return e;
    a.jn = h->wave[n];
    a.psiA = (float*)(h->ws + L.psiL[cur]);
    a.psiB = (float*)(h->ws + L.psiL[cur ^ 1]);
    if (fused) {
      // the primal and the adjoint launches of a step are independent: with
      // a side stream the adjoint runs beside the primal, and the next
      // step's restore waits for both
      cudaStream_t side = conc ? h->zs[0] : h->stream;
      if (conc) {
        if ((e = cudaEventRecord(h->zev[0], h->stream))) return e;
        if ((e = cudaStreamWaitEvent(side, h->zev[0], 0))) return e;
      }
      if ((e = smp.before(FDTD_K_REV_PRIMAL))) return e;
      if ((e = launch_rev_fused(0, rmaps[cur], a, U, h->stream))) return e;
      if ((e = smp.after(FDTD_K_REV_PRIMAL))) return e;
      if ((e = smp.before(FDTD_K_REV_ADJOINT))) return e;
      if ((e = launch_rev_fused(1, rmaps[cur], a, U, side))) return e;
      if ((e = smp.after(FDTD_K_REV_ADJOINT))) return e;
      if ((e = smp.before(FDTD_K_REV_ADJOINT_CPML))) return e;
      if ((e = launch_rev_fused(2, rmaps[cur], a, U, side))) return e;
      if ((e = launch_rev_fused(3, rmaps[cur], a, U, side))) return e;
      if ((e = smp.after(FDTD_K_REV_ADJOINT_CPML))) return e;
      if (conc) {
        if ((e = cudaEventRecord(h->zev[1], side))) return e;
        if ((e = cudaStreamWaitEvent(h->stream, h->zev[1], 0))) return e;
      }
      cur ^= 1;
      nl += 5;
      continue;
    }
    if (zg.active()) {
      const LagMaps& m = lrmaps[cur];
      if ((e = zg.fork())) return e;
      if ((e = zg.phase([&](const StepArgs& b, cudaStream_t st) {
             return launch_lag2(2, m, b, st); }, a)))
        return e;
      if ((e = zg.phase([&](const StepArgs& b, cudaStream_t st) {
             return launch_lag2(3, m, b, st); }, a)))
        return e;
      cur ^= 1;
      nl += 1 + 2 * zg.G;
      continue;
    }
    if ((e = smp.before(FDTD_K_REV_E))) return e;
    if ((e = rpair ? launch_lag2(2, lrmaps[cur], a, h->stream) : launch_rev_e(a, h->stream)))
      return e;
    if ((e = smp.after(FDTD_K_REV_E))) return e;
    if ((e = smp.before(FDTD_K_REV_H))) return e;
    if ((e = rpair ? launch_lag2(3, lrmaps[cur], a, h->stream) : launch_rev_h(a, h->stream)))
      return e;
    if ((e = smp.after(FDTD_K_REV_H))) return e;
    cur ^= 1;
    nl += 3;
  }
  if ((e = zg.join())) return e;
  *launches = nl;
  return cudaSuccess;
}

typedef cudaError_t (*EnqueueFn)(fdtd_handle*, const fdtd_record_cfg*, int*);

// Run a time loop, through a cached CUDA graph when enabled.
static int run_loop(fdtd_handle* h, const fdtd_record_cfg* rec, int dir, EnqueueFn fn,
                    int* launches, cudaEvent_t ta, cudaEvent_t tb) {
  // events for the sampled intervals exist before a capture starts
  if (h->opt_sample > 0) {
    // at most four sampled units per time step (restore, primal, two adjoint
    // launches; forward: two half-steps, record, monitor), one in m sampled
    // on average: room for twice that
    const size_t need = (size_t)(8LL * h->N / h->opt_sample) + 16;
    for (int e = 0; e < 2; ++e)
      while (h->spool[dir][e].size() < need) {
        cudaEvent_t ev;
        CK(h, cudaEventCreate(&ev));
        h->spool[dir][e].push_back(ev);
      }
  }
  CK(h, ensure_zgroups(h, dir));
  if (!h->opt_graphs) {
    CK(h, cudaEventRecord(ta, h->stream));
    cudaError_t e = fn(h, rec, launches);
    if (e) return cuda_fail(h, "time loop launch", e);
    CK(h, cudaEventRecord(tb, h->stream));
    return FDTD_OK;
  }
  GraphKey key;
  memset(&key, 0, sizeof key);
  key.dir = dir; key.dtype = rec->dtype; key.k = rec->k; key.interp = rec->interp;
  key.scaled = rec->scaled; key.kernel = h->opt_kernel; key.tile_y = h->opt_tile_y;
  key.zchunk = h->opt_zchunk;
  key.sample = h->opt_sample;
  key.stages = h->opt_stages;
  key.pdl = h->opt_pdl;
  key.prefetch = h->opt_prefetch;
  key.tile_x = h->opt_tile_x;
  key.compact = h->opt_compact;
  key.exact = h->opt_exact;
  key.coeffs = rec->coeffs;
  key.zchunk_fwd = h->opt_zchunk_fwd;
  key.zgroups = h->opt_zgroups;
  key.inject_wait = h->opt_inject_wait;
  key.reverse = h->opt_reverse;
  key.forward = h->opt_forward;
  key.zchunk_fwd2 = h->opt_zchunk_fwd2;
  key.start_buf = dir == 1 ? h->fwd_buf : 0;   // the backward starts from the forward's buffer
  auto it = h->graphs.find(key);
  if (it == h->graphs.end()) {
    cudaGraph_t graph;
    CK(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    int nl = 0;
    cudaError_t e = fn(h, rec, &nl);
    cudaError_t e2 = cudaStreamEndCapture(h->stream, &graph);
    if (e) return cuda_fail(h, "time loop capture", e);
    if (e2) return cuda_fail(h, "cudaStreamEndCapture", e2);
    cudaGraphExec_t exec;
    cudaError_t e3 = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e3) return cuda_fail(h, "cudaGraphInstantiate", e3);
    if (h->graphs.size() >= 8) drop_graphs(h);
    it = h->graphs.insert(std::make_pair(key, GraphEntry{exec, h->splan[dir]})).first;
    if (dir == 0) h->launches_fwd = nl; else h->launches_bwd = nl;
  }
  h->splan[dir] = it->second.plan;
  CK(h, cudaEventRecord(ta, h->stream));
  CK(h, cudaGraphLaunch(it->second.exec, h->stream));
  CK(h, cudaEventRecord(tb, h->stream));
  *launches = dir == 0 ? h->launches_fwd : h->launches_bwd;
  return FDTD_OK;
}

// ------------------------------------------------- device error word ---
// Status of a device error word (ERR_* bits), most specific first: an eps
// that failed validation, a bounded wait that gave up, a checked store that
// was dropped, a non-finite result.
static int err_status(unsigned err, const char** msg) {
  if (err & ERR_EPS) { *msg = "eps must be finite and >= 1"; return FDTD_ENONFINITE; }
  if (err & ERR_TIMEOUT) { *msg = "a device wait gave up (TMA pipeline)"; return FDTD_ETIMEOUT; }
  if (err & ERR_BOUNDS) {
    *msg = "bounds check: a store fell outside its buffers";
    return FDTD_ECUDA;
  }
  if (err & ERR_NONFINITE) { *msg = "a result is not finite"; return FDTD_ENONFINITE; }
  if (err) { *msg = "unknown device error bits"; return FDTD_ECUDA; }
  *msg = "";
  return FDTD_OK;
}

static int check_err(fdtd_handle* h, unsigned err) {
  const char* msg = nullptr;
  const int rc = err_status(err, &msg);
  return rc ? fail(h, rc, msg) : FDTD_OK;
}

extern "C" int fdtd_status_of_error_word(unsigned err_word) {
  const char* msg = nullptr;
  return err_status(err_word, &msg);
}

// Options that only some kernels implement, checked before a forward.
static int check_kernel_options(fdtd_handle* h) {
  if (h->opt_exact && (h->opt_kernel != 5 || h->opt_tile_y != 8 || h->opt_stages != 2 ||
                       lag_tile_x(h) != 32))
    return fail(h, FDTD_EINVAL, "exact reversal is built into kernel 5 with its default tiles");
  if (h->opt_reverse == 2 && !fused_reverse(h))
    return fail(h, FDTD_EINVAL, "the fused reverse step is built into kernel 5 with 32 x 8 tiles");
  if (h->opt_forward == 2 && !fused_forward(h))
    return fail(h, FDTD_EINVAL,
                "the fused forward step needs kernel 5, 32 x 8 tiles, CPML-free units and the "
                "source and detector outside them");
  if (h->opt_forward == 3 && !two_step_forward(h))
    return fail(h, FDTD_EINVAL,
                "the two-step forward needs kernel 5, 32 x 8 tiles, deep units and the source "
                "and detectors two cells or more away from them");
  return FDTD_OK;
}

static int forward_async(fdtd_handle* h, const float* d_eps, const fdtd_record_cfg* rec) {
  int rc = check_rec(h, rec);
  if (rc) return rc;
  if (!d_eps) return fail(h, FDTD_EINVAL, "eps is NULL");
  rc = check_kernel_options(h);
  if (rc) return rc;
  Layout L = layout_of(h, rec);
  if (!h->ws) return fail(h, FDTD_ESTATE, "no workspace bound");
  if (L.total > h->ws_bytes) return fail(h, FDTD_ENOMEM, "workspace too small for this record config");
  rc = begin(h);
  if (rc) return rc;
  h->have_forward = false;
  CK(h, cudaMemsetAsync(h->ws + L.err, 0, 256, h->stream));
  Geo g = geo_of(h);
  if (rec->dtype == kTapeBdct) CK(h, bdct_ensure_basis());
  CK(h, launch_prep(d_eps, (float*)(h->ws + L.cb), g, (unsigned*)(h->ws + L.err), h->stream));
  int nl = 0;
  nvtxRangePushA("fdtd forward loop");   // host-side range (enqueue / graph launch)
  rc = run_loop(h, rec, 0, enqueue_forward, &nl, h->t0, h->t1);
  nvtxRangePop();
  if (rc) return rc;
  h->launches_fwd = nl;
  h->fwd_buf = forward_end_buf(h);
  h->fwd_rec = *rec;
  return FDTD_OK;
}

static int forward_finish(fdtd_handle* h, double* objective) {
  Layout L = layout_of(h, &h->fwd_rec);
  h->obj_hist.assign(h->N, 0.0);
  unsigned err = 0;
  CK(h, cudaMemcpyAsync(h->obj_hist.data(), h->ws + L.obj, h->N * sizeof(double),
                        cudaMemcpyDeviceToHost, h->stream));
  std::vector<double> m(h->det2.kind ? h->N : 0);
  if (h->det2.kind)
    CK(h, cudaMemcpyAsync(m.data(), h->ws + L.obj2, h->N * sizeof(double), cudaMemcpyDeviceToHost,
                          h->stream));
  CK(h, cudaMemcpyAsync(&err, h->ws + L.err, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  h->obj2_sum = 0.0;
  for (double v : m) h->obj2_sum += v;
  CK(h, cudaEventElapsedTime(&h->fwd_ms, h->t0, h->t1));
  collect_samples(h, 0, kFwdKinds, (int)(sizeof kFwdKinds / sizeof kFwdKinds[0]));
  int rc = finish(h);
  if (rc) return rc;
  rc = check_err(h, err);
  if (rc) return rc;
  double s = 0.0;
  for (double v : h->obj_hist) s += v;
  if (!isfinite(s)) return fail(h, FDTD_ENONFINITE, "objective is not finite");
  if (objective) *objective = s;
  h->have_forward = true;
  return FDTD_OK;
}

extern "C" int fdtd_forward(fdtd_handle* h, const float* d_eps, const fdtd_record_cfg* rec,
                            double* objective) {
  if (!h) return FDTD_EINVAL;
  int rc = forward_async(h, d_eps, rec);
  if (rc) return rc;
  return forward_finish(h, objective);
}

// Upload the detectors' seeds (read by the restore kernel of every step).
// The adjoint runs with the seeds divided by a reference seed (the first
// non-zero one), so one of them is exactly 1 and the single-detector run is
// seeded exactly as without seeds; the reference multiplies the gradient in
// FP64 when it is finalised, which keeps the result exactly linear in it.
static cudaError_t upload_seeds(fdtd_handle* h, const Layout& L, double seed, double seed2,
                                cudaStream_t s) {
  if (!h->det2.kind) seed2 = 0.0;
  const double ref = seed != 0.0 ? seed : (seed2 != 0.0 ? seed2 : 1.0);
  h->seed_scale = ref;
  h->seeds[0] = seed / ref;
  h->seeds[1] = seed2 / ref;
  return cudaMemcpyAsync(h->ws + L.seeds, h->seeds, 2 * sizeof(double), cudaMemcpyHostToDevice, s);
}

static int backward_async(fdtd_handle* h, double seed, double seed2) {
  if (!h->have_forward) return fail(h, FDTD_ESTATE, "backward needs a preceding forward");
  if (layout_of(h, &h->fwd_rec).total > h->ws_bytes)
    return fail(h, FDTD_ENOMEM, "workspace too small for this record config");
  int rc = begin(h);
  if (rc) return rc;
  CK(h, upload_seeds(h, layout_of(h, &h->fwd_rec), seed, seed2, h->stream));
  int nl = 0;
  nvtxRangePushA("fdtd backward loop");
  rc = run_loop(h, &h->fwd_rec, 1, enqueue_backward, &nl, h->t2, h->t3);
  nvtxRangePop();
  if (rc) return rc;
  h->launches_bwd = nl;
  h->have_forward = false;
  // the fused reverse step leaves the reconstructed fields in the buffer of
  // the last step's output
  if (fused_reverse(h)) h->fwd_buf ^= h->N & 1;
  return FDTD_OK;
}

static int backward_finish(fdtd_handle* h, float* d_grad) {
  Layout L = layout_of(h, &h->fwd_rec);
  Geo g = geo_of(h);
  CK(h, launch_finalize((const double*)(h->ws + L.gacc), (const float*)(h->ws + L.cb), g, h->dlo,
                        h->dhi, h->seed_scale, d_grad, (unsigned*)(h->ws + L.err), h->stream));
  unsigned err = 0;
  CK(h, cudaMemcpyAsync(&err, h->ws + L.err, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  CK(h, cudaEventElapsedTime(&h->bwd_ms, h->t2, h->t3));
  collect_samples(h, 1, kBwdKinds, (int)(sizeof kBwdKinds / sizeof kBwdKinds[0]));
  int rc = finish(h);
  if (rc) return rc;
  return check_err(h, err);
}

extern "C" int fdtd_backward(fdtd_handle* h, double seed, float* d_grad_eps) {
  if (!h) return FDTD_EINVAL;
  if (!d_grad_eps) return fail(h, FDTD_EINVAL, "gradient buffer is NULL");
  int rc = backward_async(h, seed, 0.0);
  if (rc) return rc;
  return backward_finish(h, d_grad_eps);
}

extern "C" int fdtd_backward2(fdtd_handle* h, double seed, double seed2, float* d_grad_eps) {
  if (!h) return FDTD_EINVAL;
  if (!d_grad_eps) return fail(h, FDTD_EINVAL, "gradient buffer is NULL");
  if (!h->det2.kind && seed2 != 0.0) return fail(h, FDTD_ESTATE, "no second detector is set");
  int rc = backward_async(h, seed, seed2);
  if (rc) return rc;
  return backward_finish(h, d_grad_eps);
}

extern "C" int fdtd_set_detector2(fdtd_handle* h, const fdtd_detector* d) {
  if (!h) return FDTD_EINVAL;
  fdtd_detector det = {};
  if (d) det = *d;
  int dims[3] = {h->nx, h->ny, h->nz};
  if (const char* msg = detector_error(det, dims, h->P)) return fail(h, FDTD_EINVAL, msg);
  h->det2 = det;
  h->have_forward = false;
  drop_graphs(h);
  return FDTD_OK;
}

extern "C" int fdtd_objectives(const fdtd_handle* h, double* L, double* M) {
  if (!h) return FDTD_EINVAL;
  if ((int)h->obj_hist.size() != h->N) return FDTD_ESTATE;
  if (L) {
    double s = 0.0;
    for (double v : h->obj_hist) s += v;
    *L = s;
  }
  if (M) *M = h->obj2_sum;
  return FDTD_OK;
}

extern "C" int fdtd_value_and_grad_host(fdtd_handle* h, const float* h_eps,
                                        const fdtd_record_cfg* rec, double seed,
                                        double* objective, float* h_grad) {
  if (!h) return FDTD_EINVAL;
  if (!h_eps || !h_grad) return fail(h, FDTD_EINVAL, "NULL host buffer");
  if (!h->ws) return fail(h, FDTD_ESTATE, "no workspace bound");
  int rc = ensure_cuda(h);
  if (rc) return rc;
  Layout L = layout_of(h, rec ? rec : &h->fwd_rec);
  size_t n = (size_t)h->nx * h->ny * h->nz;
  size_t nd = (size_t)(h->dhi[0] - h->dlo[0]) * (h->dhi[1] - h->dlo[1]) * (h->dhi[2] - h->dlo[2]);
  CK(h, cudaEventRecord(h->ev_in, h->user_stream));
  CK(h, cudaStreamWaitEvent(h->stream, h->ev_in, 0));
  CK(h, cudaMemcpyAsync(h->ws + L.eps, h_eps, n * sizeof(float), cudaMemcpyHostToDevice,
                        h->stream));
  CK(h, cudaEventRecord(h->t4, h->stream));   // device part: after the input copy ...
  rc = fdtd_forward(h, (const float*)(h->ws + L.eps), rec, objective);
  if (rc) return rc;
  rc = backward_async(h, seed, 0.0);
  if (rc) return rc;
  rc = backward_finish(h, (float*)(h->ws + L.gout));
  if (rc) return rc;
  CK(h, cudaEventRecord(h->t5, h->stream));   // ... up to the output copy
  CK(h, cudaMemcpyAsync(h_grad, h->ws + L.gout, nd * sizeof(float), cudaMemcpyDeviceToHost,
                        h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  CK(h, cudaEventElapsedTime(&h->host_call_ms, h->t4, h->t5));
  return FDTD_OK;
}

extern "C" int fdtd_group_forward(fdtd_handle* const* hs, int n, const float* const* d_eps,
                                  const fdtd_record_cfg* rec, double* objs) {
  if (!hs || n < 0 || (n > 0 && (!d_eps || !objs))) return FDTD_EINVAL;
  for (int i = 0; i < n; ++i) {
    int rc = forward_async(hs[i], d_eps[i], rec);
    if (rc) return rc;
  }
  for (int i = 0; i < n; ++i) {
    int rc = forward_finish(hs[i], &objs[i]);
    if (rc) return rc;
  }
  return FDTD_OK;
}

extern "C" int fdtd_group_backward(fdtd_handle* const* hs, int n, const double* seeds,
                                   float* const* d_grads) {
  if (!hs || n < 0 || (n > 0 && (!seeds || !d_grads))) return FDTD_EINVAL;
  for (int i = 0; i < n; ++i) {
    if (!d_grads[i]) return fail(hs[i], FDTD_EINVAL, "gradient buffer is NULL");
    int rc = backward_async(hs[i], seeds[i], 0.0);
    if (rc) return rc;
  }
  for (int i = 0; i < n; ++i) {
    int rc = backward_finish(hs[i], d_grads[i]);
    if (rc) return rc;
  }
  return FDTD_OK;
}

// --------------------------------------------------- batched designs ----
// fdtd_batch_forward / fdtd_batch_backward: the split half-steps of every
// design run as one launch per half-step over a list of (design, tile x,
// tile y, z chunk) units, and the record and restore of every design as one
// launch per step; each CTA reads its design's own step arguments and tensor
// maps from tables in device memory.  Designs are ordered by descending step
// count, so the designs still running at a forward step, or at a reverse
// iteration t (design d runs its step N_d - 1 - t), are a prefix of the list
// and of the units.  The loops are captured once into two CUDA graphs; the
// plan (tables, graphs, stream) belongs to the first handle of the list and
// is rebuilt when the list, a workspace, an option or the record config
// changes.  The per-cell arithmetic is the split kernels', so fields and
// gradients equal those of the same designs run one by one.
struct BatchPlan {
  std::vector<size_t> sig;            // what the tables and graphs were built for
  char* dev = nullptr;                // device tables (owned)
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  int launches[2] = {0, 0};
};

static void drop_batch(fdtd_handle* h) {
  BatchPlan* b = h->batch;
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (auto& x : b->exec)
    if (x) cudaGraphExecDestroy(x);
  if (b->dev) cudaFree(b->dev);
  if (b->ev) cudaEventDestroy(b->ev);
  if (b->stream) cudaStreamDestroy(b->stream);
  delete b;
  h->batch = nullptr;
}

// The batched path runs the split half-steps and phases of kernel 5 with
// 32 x 8 tiles and two stages, one detector, no exact reversal, and an
// unscaled tape format (one thread per recorded value).
static int batch_check(fdtd_handle* const* hs, int n, const fdtd_record_cfg* rec) {
  if (!hs || n < 1 || !rec) return FDTD_EINVAL;
  for (int i = 0; i < n; ++i) {
    fdtd_handle* h = hs[i];
    if (!h) return FDTD_EINVAL;
    for (int j = 0; j < i; ++j)
      if (hs[j] == h) return fail(h, FDTD_EINVAL, "a handle appears twice in the batch");
    int rc = check_rec(h, rec);
    if (rc) return rc;
    if (!h->ws) return fail(h, FDTD_ESTATE, "no workspace bound");
    if (layout_of(h, rec).total > h->ws_bytes)
      return fail(h, FDTD_ENOMEM, "workspace too small for this record config");
    if (h->opt_kernel != 5 || fused_forward(h) || h->opt_forward == 3 || two_step_forward(h) ||
        fused_reverse(h) || lag_tile_y(h) != 8 || lag_tile_x(h) != 32 || h->opt_stages != 2 ||
        h->opt_exact || h->det2.kind || h->opt_inject_wait)
      return fail(h, FDTD_EINVAL,
                  "batched designs run kernel 5's split steps with 32 x 8 tiles, two stages, "
                  "one detector and no exact reversal");
  }
  if (rec->dtype == kTapeBdct || (rec->scaled && rec->dtype >= 2))
    return fail(hs[0], FDTD_EINVAL, "batched designs record unscaled tape formats only");
  return FDTD_OK;
}

static std::vector<size_t> batch_signature(fdtd_handle* const* hs, int n,
                                           const fdtd_record_cfg* rec) {
  std::vector<size_t> s = {(size_t)n, (size_t)rec->dtype, (size_t)rec->k, (size_t)rec->interp,
                           (size_t)rec->scaled, (size_t)rec->coeffs};
  for (int i = 0; i < n; ++i) {
    const fdtd_handle* h = hs[i];
    const size_t v[] = {(size_t)h, (size_t)h->ws, h->ws_bytes, (size_t)h->nx, (size_t)h->ny,
                        (size_t)h->nz, (size_t)h->P, (size_t)h->N, (size_t)h->opt_zchunk,
                        (size_t)(h->opt_zchunk_fwd + 1), (size_t)h->opt_zgroups,
                        (size_t)h->opt_compact, (size_t)h->opt_graphs};
    s.insert(s.end(), v, v + sizeof v / sizeof v[0]);
  }
  return s;
}

// Device copy of a host table at an aligned offset of the plan's memory.
template <class T>
static size_t batch_put(std::vector<std::pair<size_t, std::vector<char>>>& parts, size_t& off,
                        const std::vector<T>& v) {
  const size_t at = off;
  std::vector<char> bytes(v.size() * sizeof(T));
  if (!v.empty()) memcpy(bytes.data(), v.data(), bytes.size());
  off = al(off + bytes.size());
  parts.emplace_back(at, std::move(bytes));
  return at;
}

// Build, or reuse, the plan of this batch: the tables and the two captured loops.
static int batch_plan(fdtd_handle* const* hs, int n, const fdtd_record_cfg* rec,
                      BatchPlan** out) {
  fdtd_handle* h0 = hs[0];
  std::vector<size_t> sig = batch_signature(hs, n, rec);
  if (h0->batch && h0->batch->sig == sig) {
    *out = h0->batch;
    return FDTD_OK;
  }
  drop_batch(h0);
  int rc = ensure_cuda(h0);
  if (rc) return rc;
  std::vector<int> ord(n);
  for (int i = 0; i < n; ++i) ord[i] = i;
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return hs[a]->N > hs[b]->N; });
  const int maxN = hs[ord[0]]->N;
  auto active = [&](int s) {   // designs with more than s steps: a prefix of ord
    int c = 0;
    while (c < n && hs[ord[c]]->N > s) ++c;
    return c;
  };
  std::vector<LagMaps> maps(3 * (size_t)n);   // [d] forward; [n + 2d + b] reverse, aux set b
  std::vector<int4> uf, ur;
  std::vector<int> cf(n + 1, 0), cr(n + 1, 0);
  std::vector<StepArgs> bf(n), br(n);
  int rec_blocks = 0, res_blocks = 0;
  for (int d = 0; d < n; ++d) {
    fdtd_handle* h = hs[ord[d]];
    const Layout L = layout_of(h, rec);
    float* F0 = (float*)(h->ws + L.F[0]);
    float* L0 = (float*)(h->ws + L.L[0]);
    const float* cbp = (const float*)(h->ws + L.cb);
    StepArgs a = step_args(h, L);
    a.pl = L.plF;
    a.zchunk = forward_zchunk(h, a);
    a.F = F0;
    a.psiA = (float*)(h->ws + L.psiF[0]);
    a.bmap = d;
    CK(h0, encode_lag_maps(F0, F0, cbp, a.psiA, a.g, 8, 32, L.plF, &maps[d]));
    const int ntx = (h->nx + 31) / 32, nty = (h->ny + 7) / 8;
    for (int z = 0; z < (h->nz + a.zchunk - 1) / a.zchunk; ++z)
      for (int y = 0; y < nty; ++y)
        for (int x = 0; x < ntx; ++x) uf.push_back(make_int4(d, x, y, z));
    cf[d + 1] = (int)uf.size();
    bf[d] = a;
    StepArgs b = step_args(h, L);
    b.pl = L.plL;
    b.F = F0;
    b.L = L0;
    for (int k = 0; k < 2; ++k)
      CK(h0, encode_lag_maps(F0, L0, cbp, (const float*)(h->ws + L.psiL[k]), b.g, 8, 32, L.plL,
                             &maps[n + 2 * d + k]));
    for (int z = 0; z < (h->nz + b.zchunk - 1) / b.zchunk; ++z)
      for (int y = 0; y < nty; ++y)
        for (int x = 0; x < ntx; ++x) ur.push_back(make_int4(d, x, y, z));
    cr[d + 1] = (int)ur.size();
    br[d] = b;
    rec_blocks = std::max(rec_blocks, record_flat_blocks(h->faces));
    int fb, db;
    restore_blocks(h->faces, b.det, det2_of(h), &fb, &db);
    res_blocks = std::max(res_blocks, fb + db);
  }
  // per step: every running design's own arguments; record and restore jobs
  std::vector<StepArgs> af((size_t)maxN * n), ar((size_t)maxN * n);
  memset(af.data(), 0, af.size() * sizeof(StepArgs));
  memset(ar.data(), 0, ar.size() * sizeof(StepArgs));
  std::vector<RecordJob> rj;
  std::vector<int> roff(maxN + 1, 0);
  std::vector<RestoreJob> sj((size_t)maxN * n);
  memset(sj.data(), 0, sj.size() * sizeof(RestoreJob));
  const int eb = code_bytes(rec->dtype);
  for (int s = 0; s < maxN; ++s) {
    const int A = active(s);
    for (int d = 0; d < A; ++d) {
      fdtd_handle* h = hs[ord[d]];
      const Layout L = layout_of(h, rec);
      StepArgs a = bf[d];
      a.jn = h->wave[s];
      a.obj = (double*)(h->ws + L.obj) + s;
      af[(size_t)s * n + d] = a;
      const int r = (h->N - 1) % rec->k;
      if (s >= r && (s - r) % rec->k == 0) {
        const int j = (s - r) / rec->k;
        RecordJob J;
        memset(&J, 0, sizeof J);
        J.FH = J.FE = a.F;
        J.g = a.g;
        J.fc = h->faces;
        J.sample = h->ws + L.tape + (size_t)j * L.stride * eb;
        J.scale_slot = (float*)(h->ws + L.scales) + (size_t)j * 6;
        rj.push_back(J);
      }
      // reverse iteration s: design d runs its step N_d - 1 - s
      const int nd = h->N - 1 - s, cur = s & 1;
      StepArgs b = br[d];
      b.jn = h->wave[nd];
      b.psiA = (float*)(h->ws + L.psiL[cur]);
      b.psiB = (float*)(h->ws + L.psiL[cur ^ 1]);
      b.bmap = n + 2 * d + cur;
      ar[(size_t)s * n + d] = b;
      RestoreJob& R = sj[(size_t)s * n + d];
      R.F = b.F;
      R.L = b.L;
      R.g = b.g;
      R.fc = h->faces;
      R.tape = h->ws + L.tape;
      R.stride = L.stride;
      R.scales = (const float*)(h->ws + L.scales);
      interp_weights(h, rec, nd, 0, R.ip.slot[0], R.ip.w[0]);
      interp_weights(h, rec, nd, 1, R.ip.slot[1], R.ip.w[1]);
      R.det = b.det;
      R.det2 = det2_of(h);
      R.seeds = (const double*)(h->ws + L.seeds);
      restore_blocks(R.fc, R.det, R.det2, &R.face_blocks, &R.det_blocks);
    }
    roff[s + 1] = (int)rj.size();
  }
  // one device allocation for the tables (once per plan, outside the loops)
  std::vector<std::pair<size_t, std::vector<char>>> parts;
  size_t off = 0;
  const size_t o_maps = batch_put(parts, off, maps), o_uf = batch_put(parts, off, uf);
  const size_t o_ur = batch_put(parts, off, ur), o_af = batch_put(parts, off, af);
  const size_t o_ar = batch_put(parts, off, ar), o_rj = batch_put(parts, off, rj);
  const size_t o_sj = batch_put(parts, off, sj);
  BatchPlan* B = new (std::nothrow) BatchPlan();
  if (!B) return fail(h0, FDTD_ENOMEM, "batch plan");
  h0->batch = B;
  if (cudaMalloc(&B->dev, off) != cudaSuccess) {
    drop_batch(h0);
    return fail(h0, FDTD_ENOMEM, "no device memory for the batch tables");
  }
  for (auto& p : parts)
    if (!p.second.empty())
      CK(h0, cudaMemcpy(B->dev + p.first, p.second.data(), p.second.size(), cudaMemcpyHostToDevice));
  CK(h0, cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking));
  CK(h0, cudaEventCreateWithFlags(&B->ev, cudaEventDisableTiming));
  StepArgs la;   // the launch's own arguments: the lists of this launch
  memset(&la, 0, sizeof la);
  la.tile_y = 8;
  la.tile_x = 32;
  la.stages = 2;
  la.bmaps = (const LagMaps*)(B->dev + o_maps);
  LagMaps none;
  memset(&none, 0, sizeof none);
  const int dtype = rec->dtype;
  for (int dir = 0; dir < 2; ++dir) {
    CK(h0, cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    int nl = 0;
    for (int s = 0; s < maxN && !e; ++s) {
      const int A = active(s);
      if (dir == 0) {
        la.bunits = (const int4*)(B->dev + o_uf);
        la.bargs = (const StepArgs*)(B->dev + o_af) + (size_t)s * n;
        la.bcount = cf[A];
        e = launch_lag2(0, none, la, B->stream);
        if (!e && roff[s + 1] > roff[s]) {
          e = launch_record_batch(dtype, (const RecordJob*)(B->dev + o_rj) + roff[s],
                                  roff[s + 1] - roff[s], rec_blocks, B->stream);
          ++nl;
        }
        if (!e) e = launch_lag2(1, none, la, B->stream);
      } else {
        e = launch_restore_seed_batch(dtype, (const RestoreJob*)(B->dev + o_sj) + (size_t)s * n, A,
                                      res_blocks, B->stream);
        la.bunits = (const int4*)(B->dev + o_ur);
        la.bargs = (const StepArgs*)(B->dev + o_ar) + (size_t)s * n;
        la.bcount = cr[A];
        if (!e) e = launch_lag2(2, none, la, B->stream);
        if (!e) e = launch_lag2(3, none, la, B->stream);
        ++nl;
      }
      nl += 2;
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(B->stream, &graph);
    if (e || e2) {
      if (graph) cudaGraphDestroy(graph);
      drop_batch(h0);
      return cuda_fail(h0, "batched loop capture", e ? e : e2);
    }
    cudaError_t e3 = cudaGraphInstantiate(&B->exec[dir], graph, 0);
    cudaGraphDestroy(graph);
    if (e3) {
      drop_batch(h0);
      return cuda_fail(h0, "batched loop instantiate", e3);
    }
    B->launches[dir] = nl;
  }
  B->sig = sig;
  *out = B;
  return FDTD_OK;
}

// The batched loop of direction dir (0 forward, 1 backward) after every
// design's own launches, each design's stream after it.
static int batch_run(fdtd_handle* const* hs, int n, BatchPlan* B, int dir) {
  for (int i = 0; i < n; ++i) {
    CK(hs[i], cudaEventRecord(hs[i]->ev_out, hs[i]->stream));
    CK(hs[i], cudaStreamWaitEvent(B->stream, hs[i]->ev_out, 0));
  }
  for (int i = 0; i < n; ++i) CK(hs[i], cudaEventRecord(dir ? hs[i]->t2 : hs[i]->t0, B->stream));
  CK(hs[0], cudaGraphLaunch(B->exec[dir], B->stream));
  for (int i = 0; i < n; ++i) CK(hs[i], cudaEventRecord(dir ? hs[i]->t3 : hs[i]->t1, B->stream));
  CK(hs[0], cudaEventRecord(B->ev, B->stream));
  for (int i = 0; i < n; ++i) CK(hs[i], cudaStreamWaitEvent(hs[i]->stream, B->ev, 0));
  return FDTD_OK;
}

extern "C" int fdtd_batch_forward(fdtd_handle* const* hs, int n, const float* const* d_eps,
                                  const fdtd_record_cfg* rec, double* objs) {
  if (!hs || n < 1 || !d_eps || !rec || !objs) return FDTD_EINVAL;
  int rc = batch_check(hs, n, rec);
  if (rc) return rc;
  for (int i = 0; i < n; ++i) {
    if (!d_eps[i]) return fail(hs[i], FDTD_EINVAL, "eps is NULL");
    rc = check_kernel_options(hs[i]);
    if (rc) return rc;
  }
  BatchPlan* B = nullptr;
  rc = batch_plan(hs, n, rec, &B);
  if (rc) return rc;
  for (int i = 0; i < n; ++i) {   // each design's own start, on its stream
    fdtd_handle* h = hs[i];
    rc = begin(h);
    if (rc) return rc;
    h->have_forward = false;
    const Layout L = layout_of(h, rec);
    const Geo g = geo_of(h);
    CK(h, cudaMemsetAsync(h->ws + L.err, 0, 256, h->stream));
    CK(h, launch_prep(d_eps[i], (float*)(h->ws + L.cb), g, (unsigned*)(h->ws + L.err), h->stream));
    CK(h, cudaMemsetAsync(h->ws + L.F[0], 0, 6 * (size_t)g.nc * sizeof(float), h->stream));
    CK(h, cudaMemsetAsync(h->ws + L.psiF[0], 0, (size_t)L.plF.total * sizeof(float), h->stream));
    CK(h, cudaMemsetAsync(h->ws + L.obj, 0, h->N * sizeof(double), h->stream));
  }
  rc = batch_run(hs, n, B, 0);
  if (rc) return rc;
  for (int i = 0; i < n; ++i) {
    hs[i]->launches_fwd = B->launches[0];
    hs[i]->fwd_buf = 0;
    hs[i]->fwd_rec = *rec;
  }
  for (int i = 0; i < n; ++i) {
    rc = forward_finish(hs[i], &objs[i]);
    if (rc) return rc;
  }
  return FDTD_OK;
}

extern "C" int fdtd_batch_backward(fdtd_handle* const* hs, int n, const double* seeds,
                                   float* const* d_grads) {
  if (!hs || n < 1 || !seeds || !d_grads || !hs[0]) return FDTD_EINVAL;
  const fdtd_record_cfg rec = hs[0]->fwd_rec;
  for (int i = 0; i < n; ++i) {
    if (!hs[i]) return FDTD_EINVAL;
    if (!hs[i]->have_forward)
      return fail(hs[i], FDTD_ESTATE, "backward needs a preceding forward");
    if (memcmp(&hs[i]->fwd_rec, &rec, sizeof rec))
      return fail(hs[i], FDTD_EINVAL, "the batch's forwards used different record configs");
    if (!d_grads[i]) return fail(hs[i], FDTD_EINVAL, "gradient buffer is NULL");
  }
  int rc = batch_check(hs, n, &rec);
  if (rc) return rc;
  BatchPlan* B = nullptr;
  rc = batch_plan(hs, n, &rec, &B);
  if (rc) return rc;
  for (int i = 0; i < n; ++i) {
    fdtd_handle* h = hs[i];
    rc = begin(h);
    if (rc) return rc;
    const Layout L = layout_of(h, &rec);
    const size_t nc6 = 6 * (size_t)h->nz * h->ny * h->px * sizeof(float);
    const size_t psb = (size_t)L.plL.total * sizeof(float);
    const size_t nd = (size_t)(h->dhi[0] - h->dlo[0]) * (h->dhi[1] - h->dlo[1]) *
                      (h->dhi[2] - h->dlo[2]);
    CK(h, upload_seeds(h, L, seeds[i], 0.0, h->stream));
    CK(h, cudaMemsetAsync(h->ws + L.L[0], 0, nc6, h->stream));
    CK(h, cudaMemsetAsync(h->ws + L.psiL[0], 0, psb, h->stream));
    CK(h, cudaMemsetAsync(h->ws + L.psiL[1], 0, psb, h->stream));
    CK(h, cudaMemsetAsync(h->ws + L.gacc, 0, nd * sizeof(double), h->stream));
  }
  rc = batch_run(hs, n, B, 1);
  if (rc) return rc;
  for (int i = 0; i < n; ++i) {
    hs[i]->launches_bwd = B->launches[1];
    hs[i]->have_forward = false;
  }
  for (int i = 0; i < n; ++i) {
    rc = backward_finish(hs[i], d_grads[i]);
    if (rc) return rc;
  }
  return FDTD_OK;
}

extern "C" int fdtd_last_timing(const fdtd_handle* h, float* fwd_ms, float* bwd_ms,
                                int* fwd_launches, int* bwd_launches) {
  if (!h) return FDTD_EINVAL;
  if (fwd_ms) *fwd_ms = h->fwd_ms;
  if (bwd_ms) *bwd_ms = h->bwd_ms;
  if (fwd_launches) *fwd_launches = h->launches_fwd;
  if (bwd_launches) *bwd_launches = h->launches_bwd;
  return FDTD_OK;
}

extern "C" int fdtd_last_host_call_ms(const fdtd_handle* h, float* device_ms) {
  if (!h || !device_ms) return FDTD_EINVAL;
  *device_ms = h->host_call_ms;
  return FDTD_OK;
}

extern "C" int fdtd_kernel_timing(const fdtd_handle* h, int kind, float* avg_ms, int* samples) {
  if (!h || kind < 0 || kind >= FDTD_K_KINDS) return FDTD_EINVAL;
  if (avg_ms) *avg_ms = h->savg[kind];
  if (samples) *samples = h->scount[kind];
  return FDTD_OK;
}

// --------------------------------------------------------- checkpoint ---
namespace {
struct StateHeader {
  char magic[8];
  int nx, ny, nz, P, N, det2_kind;
  fdtd_record_cfg rec;
  int pad;
  long long nc, tape_bytes;
  double obj2_sum;
};
const char kStateMagic[8] = {'F', 'D', 'T', 'D', 'S', 'T', '0', '1'};

// Device regions of a forward's state for record config rec: fields, cb,
// tape, scales, objectives, second objectives (bytes each).
void state_regions(const fdtd_handle* h, const fdtd_record_cfg* rec, size_t sz[6]) {
  const Layout L = layout_of(h, rec);
  const size_t nc = (size_t)h->nz * h->ny * h->px;
  const int eb = rec->dtype == kTapeBdct ? 1 : code_bytes(rec->dtype);
  sz[0] = 6 * nc * sizeof(float);
  sz[1] = nc * sizeof(float);
  sz[2] = (size_t)L.J * L.stride * eb;
  sz[3] = (size_t)L.J * 6 * sizeof(float);
  sz[4] = (size_t)h->N * sizeof(double);
  sz[5] = (size_t)h->N * sizeof(double);
}
}  // namespace

extern "C" int fdtd_state_bytes(const fdtd_handle* h, size_t* bytes) {
  if (!h || !bytes) return FDTD_EINVAL;
  if (!h->have_forward) return FDTD_ESTATE;
  size_t sz[6];
  state_regions(h, &h->fwd_rec, sz);
  *bytes = sizeof(StateHeader) + sz[0] + sz[1] + sz[2] + sz[3] + sz[4] + sz[5];
  return FDTD_OK;
}

extern "C" int fdtd_save_state(fdtd_handle* h, void* host_buf, size_t bytes) {
  if (!h || !host_buf) return FDTD_EINVAL;
  size_t need = 0;
  if (fdtd_state_bytes(h, &need)) return fail(h, FDTD_ESTATE, "no forward state to save");
  if (bytes < need) return fail(h, FDTD_EINVAL, "state buffer too small");
  int rc = begin(h);
  if (rc) return rc;
  const Layout L = layout_of(h, &h->fwd_rec);
  size_t sz[6];
  state_regions(h, &h->fwd_rec, sz);
  StateHeader hd;
  memset(&hd, 0, sizeof hd);
  memcpy(hd.magic, kStateMagic, 8);
  hd.nx = h->nx; hd.ny = h->ny; hd.nz = h->nz; hd.P = h->P; hd.N = h->N;
  hd.det2_kind = h->det2.kind;
  hd.rec = h->fwd_rec;
  hd.nc = (long long)h->nz * h->ny * h->px;
  hd.tape_bytes = (long long)sz[2];
  hd.obj2_sum = h->obj2_sum;
  char* out = (char*)host_buf;
  memcpy(out, &hd, sizeof hd);
  out += sizeof hd;
  const size_t src[6] = {L.F[h->fwd_buf], L.cb, L.tape, L.scales, L.obj, L.obj2};
  for (int i = 0; i < 6; ++i) {
    if (i == 4) {   // the host copy of the per-step objectives
      memcpy(out, h->obj_hist.data(), sz[4]);
    } else if (sz[i]) {
      CK(h, cudaMemcpyAsync(out, h->ws + src[i], sz[i], cudaMemcpyDeviceToHost, h->stream));
    }
    out += sz[i];
  }
  CK(h, cudaStreamSynchronize(h->stream));
  return finish(h);
}

extern "C" int fdtd_load_state(fdtd_handle* h, const void* host_buf, size_t bytes) {
  if (!h || !host_buf || bytes < sizeof(StateHeader)) return FDTD_EINVAL;
  StateHeader hd;
  memcpy(&hd, host_buf, sizeof hd);
  if (memcmp(hd.magic, kStateMagic, 8) != 0) return fail(h, FDTD_EINVAL, "not a state blob");
  if (hd.nx != h->nx || hd.ny != h->ny || hd.nz != h->nz || hd.P != h->P || hd.N != h->N ||
      hd.det2_kind != h->det2.kind || hd.nc != (long long)h->nz * h->ny * h->px)
    return fail(h, FDTD_EINVAL, "state of another problem");
  int rc = check_rec(h, &hd.rec);
  if (rc) return rc;
  size_t sz[6];
  state_regions(h, &hd.rec, sz);
  if ((long long)sz[2] != hd.tape_bytes ||
      bytes < sizeof hd + sz[0] + sz[1] + sz[2] + sz[3] + sz[4] + sz[5])
    return fail(h, FDTD_EINVAL, "state blob truncated or inconsistent");
  if (!h->ws) return fail(h, FDTD_ESTATE, "no workspace bound");
  const Layout L = layout_of(h, &hd.rec);
  if (L.total > h->ws_bytes) return fail(h, FDTD_ENOMEM, "workspace too small for this state");
  rc = begin(h);
  if (rc) return rc;
  CK(h, cudaMemsetAsync(h->ws + L.err, 0, 256, h->stream));   // as a forward leaves it
  const char* in = (const char*)host_buf + sizeof hd;
  const size_t dst[6] = {L.F[0], L.cb, L.tape, L.scales, L.obj, L.obj2};
  h->obj_hist.assign(h->N, 0.0);
  for (int i = 0; i < 6; ++i) {
    if (i == 4) memcpy(h->obj_hist.data(), in, sz[4]);
    if (sz[i]) CK(h, cudaMemcpyAsync(h->ws + dst[i], in, sz[i], cudaMemcpyHostToDevice, h->stream));
    in += sz[i];
  }
  CK(h, cudaStreamSynchronize(h->stream));
  h->fwd_rec = hd.rec;
  h->fwd_buf = 0;
  h->obj2_sum = hd.obj2_sum;
  h->have_forward = true;
  return finish(h);
}

extern "C" int fdtd_read_fields(fdtd_handle* h, float* d_out) {
  if (!h || !d_out) return FDTD_EINVAL;
  if (!h->ws) return fail(h, FDTD_ESTATE, "no workspace bound");
  int rc = begin(h);
  if (rc) return rc;
  Layout L = layout_of(h, nullptr);
  CK(h, launch_gather((const float*)(h->ws + L.F[h->fwd_buf]), geo_of(h), d_out, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  return finish(h);
}

extern "C" int fdtd_objective_history(fdtd_handle* h, double* out) {
  if (!h || !out) return FDTD_EINVAL;
  if ((int)h->obj_hist.size() != h->N) return fail(h, FDTD_ESTATE, "no forward run yet");
  memcpy(out, h->obj_hist.data(), h->N * sizeof(double));
  return FDTD_OK;
}

extern "C" int fdtd_zgroup_ranges(int nch, int G, int* lo, int* hi) {
  if (nch < 1 || G < 1 || !lo || !hi) return FDTD_EINVAL;
  const int n = std::min(G, nch);
  for (int g = 0; g < n; ++g) zgroup_range(nch, n, g, &lo[g], &hi[g]);
  return n;
}

extern "C" int fdtd_deep_units(int nx, int ny, int nz, int P, int zchunk, int* box) {
  if (nx < 1 || ny < 1 || nz < 1 || P < 0 || zchunk < 1 || !box) return FDTD_EINVAL;
  Geo g;
  memset(&g, 0, sizeof g);
  g.nx = nx; g.ny = ny; g.nz = nz; g.P = P;
  const RevUnits U = deep_units(g, zchunk);
  const int v[6] = {U.ix0, U.ix1, U.iy0, U.iy1, U.iz0, U.iz1};
  for (int i = 0; i < 6; ++i) box[i] = v[i];
  return FDTD_OK;
}

extern "C" int fdtd_reverse_units(int nx, int ny, int nz, int P, int zchunk, int* counts,
                                  int* units, int max_units) {
  if (nx < 1 || ny < 1 || nz < 1 || P < 0 || zchunk < 0 || !counts) return FDTD_EINVAL;
  Geo g;
  memset(&g, 0, sizeof g);
  g.nx = nx; g.ny = ny; g.nz = nz; g.P = P;
  const RevUnits U = rev_units(g, zchunk);
  const long long np = (long long)(U.px1 - U.px0) * (U.py1 - U.py0) * (U.pz1 - U.pz0);
  const long long ni = (long long)(U.ix1 - U.ix0) * (U.iy1 - U.iy0) * (U.iz1 - U.iz0);
  const long long nall = (long long)U.ntx * U.nty * U.nzc;
  if (np > INT_MAX || nall > INT_MAX) return FDTD_EINVAL;
  counts[0] = (int)np;
  counts[1] = (int)ni;
  counts[2] = (int)(nall - ni);
  if (!units) return FDTD_OK;
  const long long n = np + nall;
  if (n > max_units) return FDTD_EINVAL;
  int* o = units;
  for (int z = U.pz0; z < U.pz1; ++z)
    for (int y = U.py0; y < U.py1; ++y)
      for (int x = U.px0; x < U.px1; ++x) { *o++ = x; *o++ = y; *o++ = z; }
  for (int z = U.iz0; z < U.iz1; ++z)
    for (int y = U.iy0; y < U.iy1; ++y)
      for (int x = U.ix0; x < U.ix1; ++x) { *o++ = x; *o++ = y; *o++ = z; }
  for (int z = 0; z < U.nzc - (U.iz1 - U.iz0); ++z)
    for (int y = 0; y < U.iy1 - U.iy0; ++y)
      for (int x = 0; x < U.ix1 - U.ix0; ++x) {
        int tx, ty, cz;
        rev_zonly_unit(U, x, y, z, &tx, &ty, &cz);
        *o++ = tx; *o++ = ty; *o++ = cz;
      }
  const long long nring = rev_ring_tiles(U) * U.nzc;
  for (long long u = 0; u < nring; ++u) {
    int tx, ty, cz;
    rev_ring_unit(U, u, &tx, &ty, &cz);
    *o++ = tx; *o++ = ty; *o++ = cz;
  }
  if (o != units + 3 * n) return FDTD_ECUDA;
  return FDTD_OK;
}

extern "C" int fdtd_selftest_wait(unsigned* d_flag, long long limit_cycles, void* cuda_stream) {
  if (!d_flag || limit_cycles <= 0) return FDTD_EINVAL;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  cudaError_t e = launch_wait_selftest(limit_cycles, d_flag, s);
  if (e) return FDTD_ECUDA;
  unsigned flag = 0;
  if (cudaMemcpyAsync(&flag, d_flag, sizeof flag, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return FDTD_ECUDA;
  return (flag & ERR_TIMEOUT) ? FDTD_ETIMEOUT : FDTD_OK;
}

extern "C" int fdtd_encode(int dtype, int scaled, const float* d_in, size_t n, void* d_code,
                           float* d_scale, void* cuda_stream) {
  if (dtype < 0 || dtype >= kTapeDtypes || !d_in || !d_code || !d_scale) return FDTD_EINVAL;
  if (scaled && dtype < 2) return FDTD_EINVAL;
  cudaError_t e = launch_encode(dtype, scaled, d_in, n, d_code, d_scale, (cudaStream_t)cuda_stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)cuda_stream);
  return e == cudaSuccess ? FDTD_OK : FDTD_ECUDA;
}

extern "C" int fdtd_bdct_encode(const float* d_in, int nu, int nv, int coeffs,
                                signed char* d_codes, float* d_scales, void* cuda_stream) {
  if (!d_in || !d_codes || !d_scales || nu < 1 || nv < 1 || coeffs < 1 || coeffs > 64)
    return FDTD_EINVAL;
  cudaError_t e = bdct_ensure_basis();
  if (e == cudaSuccess)
    e = launch_bdct_encode(d_in, nu, nv, coeffs, d_codes, d_scales, (cudaStream_t)cuda_stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)cuda_stream);
  return e == cudaSuccess ? FDTD_OK : FDTD_ECUDA;
}

extern "C" int fdtd_bdct_basis(float* out) {
  if (!out) return FDTD_EINVAL;
  bdct_basis_host(out);
  return FDTD_OK;
}

extern "C" int fdtd_bdct_decode(const signed char* d_codes, const float* d_scales, int nu, int nv,
                                int coeffs, float* d_out, void* cuda_stream) {
  if (!d_codes || !d_scales || !d_out || nu < 1 || nv < 1 || coeffs < 1 || coeffs > 64)
    return FDTD_EINVAL;
  cudaError_t e = bdct_ensure_basis();
  if (e == cudaSuccess)
    e = launch_bdct_decode(d_codes, d_scales, nu, nv, coeffs, d_out, (cudaStream_t)cuda_stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)cuda_stream);
  return e == cudaSuccess ? FDTD_OK : FDTD_ECUDA;
}

extern "C" int fdtd_decode(int dtype, const void* d_code, size_t n, const float* d_scale,
                           float* d_out, void* cuda_stream) {
  if (dtype < 0 || dtype >= kTapeDtypes || !d_code || !d_scale || !d_out) return FDTD_EINVAL;
  cudaError_t e = launch_decode(dtype, d_code, n, d_scale, d_out, (cudaStream_t)cuda_stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)cuda_stream);
  return e == cudaSuccess ? FDTD_OK : FDTD_ECUDA;
}

// ------------------------------------------------ no-allocation variant ---
// A fixed scratch area compiled into the library stands in for the caller's
// workspace.  Host code must not use g_noalloc_scratch's name as a device
// address (it is a host-side stand-in); the address comes from
// cudaGetSymbolAddress, looked up once per device with that device current.
static __device__ __align__(256) unsigned char g_noalloc_scratch[FDTD_NOALLOC_SCRATCH_BYTES];

static void* g_noalloc_ptr[256];
static std::mutex g_noalloc_mu;

static int noalloc_scratch(fdtd_handle* h, void** out) {
  int dev = 0;
  CK(h, cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) return fail(h, FDTD_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return cuda_fail(h, "cudaGetSymbolAddress(noalloc scratch)", e);
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return FDTD_OK;
}

extern "C" int fdtd_value_and_grad_noalloc(fdtd_handle* h, const float* d_eps,
                                           const fdtd_record_cfg* rec, double seed,
                                           double* objective, float* d_grad) {
  if (!h) return FDTD_EINVAL;
  int rc = check_rec(h, rec);
  if (rc) return rc;
  if (!d_eps || !d_grad) return fail(h, FDTD_EINVAL, "NULL device buffer");
  rc = check_kernel_options(h);
  if (rc) return rc;
  Layout L = layout_of(h, rec);
  if (L.total > FDTD_NOALLOC_SCRATCH_BYTES) {
    char buf[256];
    snprintf(buf, sizeof buf,
             "problem needs a %zu-byte workspace; the fixed no-allocation scratch holds %llu bytes",
             L.total, (unsigned long long)FDTD_NOALLOC_SCRATCH_BYTES);
    return fail(h, FDTD_ENOMEM, buf);
  }
  void* scratch = nullptr;
  rc = noalloc_scratch(h, &scratch);
  if (rc) return rc;

  // Run the usual time loops on the caller's stream with the scratch as the
  // workspace: direct launches (no graph), no sampling events, one stream.
  char* ws0 = h->ws;
  size_t b0 = h->ws_bytes;
  bool up0 = h->tables_uploaded;
  cudaStream_t s0 = h->stream;
  int samp0 = h->opt_sample, zg0 = h->opt_zgroups;   // no side streams here
  h->ws = (char*)scratch;
  h->ws_bytes = FDTD_NOALLOC_SCRATCH_BYTES;
  h->stream = h->user_stream;
  h->opt_sample = 0;
  h->opt_zgroups = 1;
  h->have_forward = false;
  auto restore = [&]() {
    h->ws = ws0;
    h->ws_bytes = b0;
    h->tables_uploaded = up0;
    h->stream = s0;
    h->opt_sample = samp0;
    h->opt_zgroups = zg0;
    h->have_forward = false;
  };
  auto run = [&]() -> int {
    cudaStream_t s = h->stream;
    Layout L0 = layout_of(h, nullptr);
    CK(h, cudaMemcpyAsync(h->ws + L0.prof, h->prof.data(), h->prof.size() * sizeof(float),
                          cudaMemcpyHostToDevice, s));
    if (!h->srcw.empty())
      CK(h, cudaMemcpyAsync(h->ws + L0.srcw, h->srcw.data(), h->srcw.size() * sizeof(float),
                            cudaMemcpyHostToDevice, s));
    CK(h, cudaMemsetAsync(h->ws + L.err, 0, 256, s));
    Geo g = geo_of(h);
    if (rec->dtype == kTapeBdct) CK(h, bdct_ensure_basis());
    CK(h, launch_prep(d_eps, (float*)(h->ws + L.cb), g, (unsigned*)(h->ws + L.err), s));
    int nl = 0;
    cudaError_t e = enqueue_forward(h, rec, &nl);
    if (e) return cuda_fail(h, "forward launch", e);
    h->fwd_buf = forward_end_buf(h);
    // objective: per-step slots summed on the host in chunks
    double sum = 0.0, chunk[256];
    for (int n0 = 0; n0 < h->N; n0 += 256) {
      int m = h->N - n0 < 256 ? h->N - n0 : 256;
      CK(h, cudaMemcpyAsync(chunk, h->ws + L.obj + (size_t)n0 * sizeof(double),
                            m * sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(h, cudaStreamSynchronize(s));
      for (int i = 0; i < m; ++i) sum += chunk[i];
    }
    unsigned err = 0;
    CK(h, cudaMemcpyAsync(&err, h->ws + L.err, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    CK(h, cudaStreamSynchronize(s));
    int rc2 = check_err(h, err);
    if (rc2) return rc2;
    if (!isfinite(sum)) return fail(h, FDTD_ENONFINITE, "objective is not finite");
    CK(h, upload_seeds(h, L, seed, 0.0, s));
    e = enqueue_backward(h, rec, &nl);
    if (e) return cuda_fail(h, "backward launch", e);
    CK(h, launch_finalize((const double*)(h->ws + L.gacc), (const float*)(h->ws + L.cb), g,
                          h->dlo, h->dhi, h->seed_scale, d_grad, (unsigned*)(h->ws + L.err), s));
    CK(h, cudaMemcpyAsync(&err, h->ws + L.err, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    CK(h, cudaStreamSynchronize(s));
    rc2 = check_err(h, err);
    if (rc2) return rc2;
    if (objective) *objective = sum;
    return FDTD_OK;
  };
  rc = run();
  restore();
  return rc;
}
