// Host side of the C ABI: argument checks, Nystrom rule tables, support-point
// geometry, pair classification, device memory and the stage launches.
#include <cuda_runtime.h>
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <map>
#include <mutex>
#include <thread>
#include <tuple>
#include <vector>

#include "mueller.h"
#include "green.cuh"
#include "lu.cuh"
#include "fields.cuh"
#include "mixed.cuh"
#include "ozaki.cuh"

static thread_local std::string g_err;
static int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}
#define CK(x)                                                                                   \
  do {                                                                                          \
    cudaError_t e_ = (x);                                                                       \
    if (e_ != cudaSuccess) return fail(MUELLER_ECUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)

static cd tocd(mueller_c128 a) { return cd{a.re, a.im}; }

// ---------------------------------------------------------------- rules (Section 5)
// Gauss-Legendre nodes (increasing) and weights on [-1, 1] by Newton's method
// on the three-term recurrence of P_n.
static void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0); w.assign(n, 0.0);
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double t = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = t;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
        p0 = p1; p1 = p2;
      }
      dp = n * (t * p1 - p0) / (t * t - 1.0);
      double dt = p1 / dp;
      t -= dt;
      if (std::fabs(dt) < 1e-16) {
        p0 = 1.0; p1 = t;
        for (int k = 2; k <= n; ++k) {
          double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
          p0 = p1; p1 = p2;
        }
        dp = n * (t * p1 - p0) / (t * t - 1.0);
        break;
      }
    }
    x[i] = -t; x[n - 1 - i] = t;
    double wi = 2.0 / ((1.0 - t * t) * dp * dp);
    w[i] = wi; w[n - 1 - i] = wi;
  }
}

struct Rules {
  std::vector<double> x16, w16, bary;   // panel nodes, weights, barycentric weights
  std::vector<double> self_u, self_w;   // reference self rule on [0, 1]
  std::vector<double> adj_u, adj_w;     // reference adjacent rule on [0, 1] at corners (graded composite)
  std::vector<double> adjs_u, adjs_w;   // reference adjacent rule on [0, 1] at smooth junctions
};

// Reference rule on [0, 1] graded toward 0: intervals [4^-(j+1), 4^-j] and
// the innermost [0, 4^-levels], ng Gauss points each.
static void graded_rule(int levels, int ng, std::vector<double>& u, std::vector<double>& w) {
  std::vector<double> x, wx;
  gauss_legendre(ng, x, wx);
  u.clear(); w.clear();
  for (int j = 0; j <= levels; ++j) {
    const double a = j < levels ? std::pow(4.0, -(j + 1)) : 0.0, b = std::pow(4.0, -j);
    for (int q = 0; q < ng; ++q) {
      u.push_back(0.5 * (a + b) + 0.5 * (b - a) * x[q]);
      w.push_back(0.5 * (b - a) * wx[q]);
    }
  }
}

static Rules make_rules() {
  Rules R;
  gauss_legendre(P_NODES, R.x16, R.w16);
  R.bary.resize(P_NODES);
  for (int k = 0; k < P_NODES; ++k)
    R.bary[k] = ((k % 2) ? -1.0 : 1.0) * std::sqrt((1.0 - R.x16[k] * R.x16[k]) * R.w16[k]);
  R.self_u.assign(MUELLER_SELF_U, MUELLER_SELF_U + MUELLER_SELF_SIDE);
  R.self_w.assign(MUELLER_SELF_W, MUELLER_SELF_W + MUELLER_SELF_SIDE);
  graded_rule(5, 16, R.adj_u, R.adj_w);
  R.adjs_u.assign(MUELLER_ADJ_U, MUELLER_ADJ_U + MUELLER_ADJ_SMOOTH);
  R.adjs_w.assign(MUELLER_ADJ_W, MUELLER_ADJ_W + MUELLER_ADJ_SMOOTH);
  return R;
}

// initialised once, thread-safely (concurrent builds on several streams)
static const Rules& rules() {
  static const Rules R = make_rules();
  return R;
}

// Lagrange basis at t through the 16 panel nodes (barycentric form).
static void lagrange_row(const Rules& R, double t, double* L) {
  for (int k = 0; k < P_NODES; ++k)
    if (std::fabs(t - R.x16[k]) < 1e-300) {
      for (int j = 0; j < P_NODES; ++j) L[j] = (j == k) ? 1.0 : 0.0;
      return;
    }
  double den = 0.0;
  for (int k = 0; k < P_NODES; ++k) {
    L[k] = R.bary[k] / (t - R.x16[k]);
    den += L[k];
  }
  for (int k = 0; k < P_NODES; ++k) L[k] /= den;
}

// ---------------------------------------------------------------- setup
struct Setup {
  int N = 0, n = 0, nP = 0, closed = 0, M = 0, nphi = 0, formulation = 0, precision = 0;
  double omega = 0, split_eps = 1e-17, rmax = 0, refine_tol = 1e-14;
  int refine_max_iter = 10;
  cd k0{}, k1{}, eps0{}, mu0{}, eps1{}, mu1{};
  std::vector<double> r, z, rp, zp, w, sw;                  // nodes
  std::vector<double> sr, sz, srp, szp, sW;                 // support points
  std::vector<double> sdr, sdz;                             // own-panel: target - point
  std::vector<double> Lself, Ladj;
  std::vector<int> adj_rule, adj_n;    // [nP][2]: rule (0 smooth, 1 corner) and point count of each panel end
  std::vector<int> split_far, split_sup;
  std::vector<double> split_pairs;                          // [n_split][4]
  long long n_far = 0, n_sup = 0;
  GreenParams gp{};
  AsmParams ap{};
  cd sE{}, sH{};
};

static bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

static cd csqrt_im_nonneg(cd z) {
  cd s = csqrt_principal(z);
  if (s.y < 0) s = -s;
  return s;
}

static int nphi_needed(int M, double kmax, double rmax, int nphi_req) {
  double a = 2.0 * kmax * rmax;
  int Na = (int)std::ceil((a + 10.0 * std::cbrt(a) + 10.0) / 2.0) + 2;
  int need = 2 * (M + 2 + Na);
  int v = std::max(16, nphi_req > 0 ? nphi_req : 16);
  while (v < need && v < (1 << 24)) v *= 2;  // beyond any shared-memory limit; rejected by the caller
  if (!is_pow2(v)) {
    int p = 16;
    while (p < v) p *= 2;
    v = p;
  }
  return v;
}

static void fill_green_params(GreenParams& gp, int M, int nphi, cd k0, cd k1) {
  gp.M = M; gp.Ms = M + 2; gp.nphi = nphi; gp.H = nphi / 2 + 1; gp.Mq = nphi / 2 - 1;
  gp.kp0 = kpow(k0); gp.kp1 = kpow(k1);
  gp.gamma0 = -0.25 * (k0 * k0 - k1 * k1);
  gp.k0_real = k0.y == 0.0; gp.k1_real = k1.y == 0.0;
  gp.qmax = (nphi - 1) / 8;  // grid ladder 16, 24, .., below nphi (multiples of 8: two folds)
}

// Split decision: the plain trapezoid's aliasing zeta^(nphi-M-1) is above eps,
// with zeta = e^{-l}, l = acosh(chi), chi = 1 + d^2 / (2 r_t r_s).  Since l
// grows with chi, (nphi-M-1) l < -ln eps is chi - 1 < cosh(l_max) - 1 with
// l_max = -ln(eps) / (nphi-M-1): a threshold on d^2 / (2 r_t r_s) fixed per build.
struct SplitTest {
  double cthr;  // cosh(l_max) - 1 = 2 sinh^2(l_max / 2); +inf when nphi <= M + 1
  SplitTest(int nphi, int M, double eps) {
    const int span = nphi - M - 1;
    if (span <= 0) { cthr = HUGE_VAL; return; }
    const double sh = std::sinh(0.5 * (-std::log(eps) / span));
    cthr = 2.0 * sh * sh;
  }
  bool operator()(double rt, double dr, double dz) const {
    const double d2 = dr * dr + dz * dz, B = 2.0 * rt * (rt - dr);
    return d2 < cthr * B;
  }
};

// Runs body(lo, hi) over [0, count) in contiguous chunks on up to 16 host threads.
template <class F>
static void parallel_chunks(int count, const F& body) {
  const int hw = (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  const int nt = std::max(1, std::min(hw, count / 4));
  if (nt == 1) { body(0, count); return; }
  std::vector<std::thread> th;
  for (int t = 0; t < nt; ++t) {
    const int lo = (int)((long long)count * t / nt), hi = (int)((long long)count * (t + 1) / nt);
    th.emplace_back([&body, lo, hi] { body(lo, hi); });
  }
  for (auto& x : th) x.join();
}

static int setup_inputs(const mueller_curve* cv, const mueller_media* md, int M, const mueller_options* op,
                        Setup& S) {
  if (!cv || !md || !op) return fail(MUELLER_EINVAL, "null argument");
  if (cv->n_panels < 1) return fail(MUELLER_EINVAL, "n_panels must be >= 1");
  if (cv->closed && cv->n_panels < 3) return fail(MUELLER_EINVAL, "closed curves need >= 3 panels");
  if (!cv->r || !cv->z || !cv->dr || !cv->dz) return fail(MUELLER_EINVAL, "null curve array");
  if (M < 0 || M > 4096) return fail(MUELLER_EINVAL, "M out of range [0, 4096]");
  if (op->formulation != 0 && op->formulation != 1) return fail(MUELLER_EINVAL, "formulation must be 0 or 1");
  if (op->precision < 0 || op->precision > 2)
    return fail(MUELLER_EINVAL, "precision must be 0 (FP64), 1 (mixed, tensor-core residuals) or 2 (mixed, FP64 residuals)");
  if (op->precision != 0 && !(op->refine_tol > 0.0 && op->refine_tol < 1.0))
    return fail(MUELLER_EINVAL, "mixed precision needs 0 < refine_tol < 1");
  if (!(md->omega > 0.0)) return fail(MUELLER_EINVAL, "omega must be > 0 (the method excludes omega -> 0)");
  auto ok_body = [](mueller_c128 v) { return v.re > 0.0 && v.im >= 0.0; };
  auto ok_back = [](mueller_c128 v) { return v.re > 0.0 && v.im == 0.0; };
  if (!ok_back(md->eps0) || !ok_back(md->mu0)) return fail(MUELLER_EINVAL, "eps0, mu0 must be real and > 0");
  if (!ok_body(md->eps1) || !ok_body(md->mu1))
    return fail(MUELLER_EINVAL, "eps1, mu1 need Re > 0 and Im >= 0 (eq. materials)");
  const Rules& R = rules();
  S.nP = cv->n_panels; S.N = 16 * S.nP; S.n = 4 * S.N; S.closed = cv->closed ? 1 : 0; S.M = M;
  S.formulation = op->formulation; S.precision = op->precision;
  S.refine_tol = op->refine_tol; S.refine_max_iter = op->refine_max_iter > 0 ? op->refine_max_iter : 10;
  S.split_eps = op->split_eps > 0 ? op->split_eps : 1e-17;
  S.omega = md->omega;
  S.eps0 = tocd(md->eps0); S.mu0 = tocd(md->mu0); S.eps1 = tocd(md->eps1); S.mu1 = tocd(md->mu1);
  S.k0 = md->omega * csqrt_im_nonneg(S.eps0 * S.mu0);
  S.k1 = md->omega * csqrt_im_nonneg(S.eps1 * S.mu1);
  const int N = S.N;
  S.r.assign(cv->r, cv->r + N); S.z.assign(cv->z, cv->z + N);
  S.rp.resize(N); S.zp.resize(N); S.w.resize(N); S.sw.resize(N);
  double area = 0.0;
  S.rmax = 0.0;
  for (int i = 0; i < N; ++i) {
    double sp = std::hypot(cv->dr[i], cv->dz[i]);
    if (!(cv->r[i] > 0.0)) return fail(MUELLER_EINVAL, "curve nodes need r > 0");
    if (!(sp > 0.0)) return fail(MUELLER_EINVAL, "curve has a zero tangent at a node");
    S.rp[i] = cv->dr[i] / sp; S.zp[i] = cv->dz[i] / sp;
    S.w[i] = R.w16[i % P_NODES] * sp;
    S.sw[i] = std::sqrt(S.w[i]);
    area += 0.5 * R.w16[i % P_NODES] * (cv->r[i] * cv->dz[i] - cv->z[i] * cv->dr[i]);
    S.rmax = std::max(S.rmax, cv->r[i]);
  }
  if (!(area > 0.0))
    return fail(MUELLER_EINVAL, "curve must run counterclockwise in (r, z) (outward normal n = (z', -r'))");
  double kmax = std::max(cabs(S.k0), cabs(S.k1));
  S.nphi = nphi_needed(M, kmax, S.rmax, op->n_phi);
  fill_green_params(S.gp, M, S.nphi, S.k0, S.k1);
  if (!green_fits_smem(S.gp))
    return fail(MUELLER_EINVAL, "n_phi (" + std::to_string(S.nphi) + ") and M need more shared memory per warp "
                "than a CTA can have");
  // block coefficients
  cd iw = C(0.0, S.omega);
  AsmParams& ap = S.ap;
  ap.k0sq = S.k0 * S.k0; ap.k1sq = S.k1 * S.k1;
  if (S.formulation == 0) {
    ap.aEJ = C(1.0); ap.aHM = C(-1.0);
    ap.cEM0 = -(iw * S.eps0); ap.cEM1 = iw * S.eps1;
    ap.cHJ0 = -(iw * S.mu0); ap.cHJ1 = iw * S.mu1;
    ap.dEM = 0.5 * (iw * (S.eps0 + S.eps1)); ap.dHJ = 0.5 * (iw * (S.mu0 + S.mu1));
    S.sE = iw * S.eps0; S.sH = iw * S.mu0;
  } else {
    ap.aEJ = S.mu0 / S.eps0; ap.aHM = -(S.eps0 / S.mu0);
    ap.cEM0 = -(iw * S.mu0); ap.cEM1 = iw * S.mu1;
    ap.cHJ0 = -(iw * S.eps0); ap.cHJ1 = iw * S.eps1;
    ap.dEM = -0.5 * (iw * (S.mu0 + S.mu1)); ap.dHJ = -0.5 * (iw * (S.eps0 + S.eps1));
    S.sE = iw * S.mu0; S.sH = iw * S.eps0;
  }
  // the far-pair assembly drops the products by zero parts when these hold exactly
  ap.simple = ap.k0sq.y == 0.0 && ap.k1sq.y == 0.0 && ap.cEM0.x == 0.0 && ap.cEM1.x == 0.0 && ap.cHJ0.x == 0.0 &&
              ap.cHJ1.x == 0.0 && ap.aEJ.x == 1.0 && ap.aEJ.y == 0.0 && ap.aHM.x == -1.0 && ap.aHM.y == 0.0;
  return MUELLER_OK;
}

// Support points and interpolation tables (eq. eq_nyslike2).
static void setup_support(const mueller_curve* cv, Setup& S) {
  const Rules& R = rules();
  const int ns = (int)R.self_u.size();
  S.Lself.assign((size_t)P_NODES * SELF_PTS * P_NODES, 0.0);
  std::vector<double> tau_self((size_t)P_NODES * SELF_PTS), wt_self((size_t)P_NODES * SELF_PTS);
  for (int a = 0; a < P_NODES; ++a) {
    double ti = R.x16[a], Lm = ti + 1.0, Lp = 1.0 - ti;
    for (int s = 0; s < ns; ++s) {
      tau_self[a * SELF_PTS + s] = ti - Lm * R.self_u[s];
      wt_self[a * SELF_PTS + s] = Lm * R.self_w[s];
      tau_self[a * SELF_PTS + ns + s] = ti + Lp * R.self_u[s];
      wt_self[a * SELF_PTS + ns + s] = Lp * R.self_w[s];
    }
    for (int s = 0; s < SELF_PTS; ++s)
      lagrange_row(R, tau_self[a * SELF_PTS + s], &S.Lself[((size_t)a * SELF_PTS + s) * P_NODES]);
  }
  // neighbouring panels: per rule (0 smooth junction, 1 corner) and panel end
  // (0: tau = -1, 1: tau = +1), points tau = -1 + 2u or 1 - 2u
  std::vector<double> tau_adj(4 * ADJ_PTS, 0.0), wt_adj(4 * ADJ_PTS, 0.0);
  S.Ladj.assign((size_t)4 * ADJ_PTS * P_NODES, 0.0);
  for (int rule = 0; rule < 2; ++rule) {
    const std::vector<double>& u = rule ? R.adj_u : R.adjs_u;
    const std::vector<double>& w = rule ? R.adj_w : R.adjs_w;
    for (int e = 0; e < 2; ++e)
      for (size_t s = 0; s < u.size(); ++s) {
        const size_t k = (size_t)(rule * 2 + e) * ADJ_PTS + s;
        tau_adj[k] = e == 0 ? -1.0 + 2.0 * u[s] : 1.0 - 2.0 * u[s];
        wt_adj[k] = 2.0 * w[s];
        lagrange_row(R, tau_adj[k], &S.Ladj[k * P_NODES]);
      }
  }
  // junction j joins panel j's end +1 and panel j+1's end -1 (the last one
  // wraps for closed curves): a corner when the two end tangents, from the
  // panels' degree-15 interpolants of (dr, dz), differ by more than 10 degrees
  std::vector<double> Lm1(P_NODES), Lp1(P_NODES);
  lagrange_row(R, -1.0, Lm1.data());
  lagrange_row(R, 1.0, Lp1.data());
  auto tangent = [&](int Q, const std::vector<double>& L, double* t) {
    t[0] = t[1] = 0.0;
    for (int k = 0; k < P_NODES; ++k) { t[0] += L[k] * cv->dr[Q * P_NODES + k]; t[1] += L[k] * cv->dz[Q * P_NODES + k]; }
  };
  const int wrap = S.closed && S.nP > 2;
  S.adj_rule.assign((size_t)2 * S.nP, -1);
  S.adj_n.assign((size_t)2 * S.nP, 0);
  for (int j = 0; j < S.nP - 1 + wrap; ++j) {
    const int A = j, B = (j + 1) % S.nP;
    double ta[2], tb[2];
    tangent(A, Lp1, ta);
    tangent(B, Lm1, tb);
    const double c = (ta[0] * tb[0] + ta[1] * tb[1]) / (std::hypot(ta[0], ta[1]) * std::hypot(tb[0], tb[1]));
    const int rule = c < 0.98480775301220806 ? 1 : 0;  // cos 10 degrees
    const int n = rule ? (int)R.adj_u.size() : (int)R.adjs_u.size();
    S.adj_rule[2 * A + 1] = rule; S.adj_n[2 * A + 1] = n;
    S.adj_rule[2 * B + 0] = rule; S.adj_n[2 * B + 0] = n;
  }
  const size_t npts = (size_t)S.nP * PTS_PER_PANEL;
  S.sr.resize(npts); S.sz.resize(npts); S.srp.resize(npts); S.szp.resize(npts); S.sW.resize(npts);
  S.sdr.assign(npts, 0.0); S.sdz.assign(npts, 0.0);
  parallel_chunks(S.nP, [&](int q_lo, int q_hi) {
  for (int Q = q_lo; Q < q_hi; ++Q) {
    const double* r = cv->r + Q * P_NODES;
    const double* z = cv->z + Q * P_NODES;
    const double* dr = cv->dr + Q * P_NODES;
    const double* dz = cv->dz + Q * P_NODES;
    for (int t = 0; t < PTS_PER_PANEL; ++t) {
      const double* L;
      double wt;
      if (t < P_NODES * SELF_PTS) { L = &S.Lself[(size_t)t * P_NODES]; wt = wt_self[t]; }
      else {
        const int e = (t - P_NODES * SELF_PTS) / ADJ_PTS, s = (t - P_NODES * SELF_PTS) % ADJ_PTS;
        const int rule = S.adj_rule[2 * Q + e];
        if (rule < 0 || s >= S.adj_n[2 * Q + e]) {  // no neighbour at this end, or beyond the rule's points
          const size_t id = (size_t)Q * PTS_PER_PANEL + t;
          S.sr[id] = S.sz[id] = S.srp[id] = S.szp[id] = S.sW[id] = 0.0;
          continue;
        }
        const size_t k = (size_t)(rule * 2 + e) * ADJ_PTS + s;
        L = &S.Ladj[k * P_NODES]; wt = wt_adj[k];
      }
      double vr = 0, vz = 0, vdr = 0, vdz = 0;
      for (int k = 0; k < P_NODES; ++k) {
        vr += L[k] * r[k]; vz += L[k] * z[k]; vdr += L[k] * dr[k]; vdz += L[k] * dz[k];
      }
      double sp = std::hypot(vdr, vdz);
      size_t id = (size_t)Q * PTS_PER_PANEL + t;
      S.sr[id] = vr; S.sz[id] = vz; S.srp[id] = vdr / sp; S.szp[id] = vdz / sp; S.sW[id] = wt * sp;
      if (t < P_NODES * SELF_PTS) {
        // own-panel point of target a: x_t - x_s = -sum_{k != a} L_k(tau_s) (x_k - x_a)
        int a = t / SELF_PTS;
        double ddr = 0.0, ddz = 0.0;
        for (int k = 0; k < P_NODES; ++k) {
          if (k == a) continue;
          ddr -= L[k] * (r[k] - r[a]);
          ddz -= L[k] * (z[k] - z[a]);
        }
        S.sdr[id] = ddr; S.sdz[id] = ddz;
      }
    }
  }
  });
}

static bool near_panels_h(int Pi, int Pj, int nP, int closed) {
  int d = Pi - Pj;
  if (d >= -1 && d <= 1) return true;
  if (closed && nP > 2 && (d == nP - 1 || d == -(nP - 1))) return true;
  return false;
}

static long long support_pid(const Setup& S, int i, int slot) {
  int P = i / P_NODES, loc = i % P_NODES;
  if (slot < SELF_PTS) return (long long)P * PTS_PER_PANEL + loc * SELF_PTS + slot;
  if (slot < SELF_PTS + ADJ_PTS) {
    int Q = P - 1;
    if (Q < 0) { if (!S.closed) return -1; Q = S.nP - 1; }
    if (slot - SELF_PTS >= S.adj_n[2 * Q + 1]) return -1;  // beyond the rule of Q's end +1
    return (long long)Q * PTS_PER_PANEL + P_NODES * SELF_PTS + ADJ_PTS + (slot - SELF_PTS);
  }
  int Q = P + 1;
  if (Q >= S.nP) { if (!S.closed) return -1; Q = 0; }
  if (slot - SELF_PTS - ADJ_PTS >= S.adj_n[2 * Q + 0]) return -1;  // beyond the rule of Q's end -1
  return (long long)Q * PTS_PER_PANEL + P_NODES * SELF_PTS + (slot - SELF_PTS - ADJ_PTS);
}

// Split pairs get ids in a fixed order: far pairs (i, j) row-major, then
// support pairs (i, slot) row-major.  Rows are classified on host threads
// (flags and per-row counts), then numbered from the prefix sums.
static void setup_pairs(Setup& S) {
  const int N = S.N;
  const SplitTest split(S.nphi, S.M, S.split_eps);
  S.split_far.assign((size_t)N * N, -1);
  S.split_sup.assign((size_t)N * NEAR_SLOTS, -1);
  std::vector<long long> cnt_far(N + 1, 0), cnt_sup(N + 1, 0), nfar(N, 0), nsup(N, 0);
  auto sup_disp = [&](int i, int slot, long long pid, double* dr, double* dz) {
    if (slot < SELF_PTS) { *dr = S.sdr[pid]; *dz = S.sdz[pid]; }
    else { *dr = S.r[i] - S.sr[pid]; *dz = S.z[i] - S.sz[pid]; }
  };
  parallel_chunks(N, [&](int lo, int hi) {
    for (int i = lo; i < hi; ++i) {
      long long cf = 0, cs = 0;
      for (int j = 0; j < N; ++j) {
        if (near_panels_h(i / P_NODES, j / P_NODES, S.nP, S.closed)) continue;
        ++nfar[i];
        if (split(S.r[i], S.r[i] - S.r[j], S.z[i] - S.z[j])) { S.split_far[(size_t)i * N + j] = 0; ++cf; }
      }
      for (int slot = 0; slot < NEAR_SLOTS; ++slot) {
        long long pid = support_pid(S, i, slot);
        if (pid < 0) continue;
        ++nsup[i];
        double dr, dz;
        sup_disp(i, slot, pid, &dr, &dz);
        if (split(S.r[i], dr, dz)) { S.split_sup[(size_t)i * NEAR_SLOTS + slot] = 0; ++cs; }
      }
      cnt_far[i + 1] = cf;
      cnt_sup[i + 1] = cs;
    }
  });
  for (int i = 0; i < N; ++i) cnt_far[i + 1] += cnt_far[i];
  cnt_sup[0] = cnt_far[N];
  for (int i = 0; i < N; ++i) cnt_sup[i + 1] += cnt_sup[i];
  S.n_far = 0; S.n_sup = 0;
  for (int i = 0; i < N; ++i) { S.n_far += nfar[i]; S.n_sup += nsup[i]; }
  S.split_pairs.assign((size_t)cnt_sup[N] * 4, 0.0);
  parallel_chunks(N, [&](int lo, int hi) {
    for (int i = lo; i < hi; ++i) {
      long long id = cnt_far[i];
      for (int j = 0; j < N; ++j) {
        int& f = S.split_far[(size_t)i * N + j];
        if (f < 0) continue;
        f = (int)id;
        const double v[4] = {S.r[i], S.z[i], S.r[i] - S.r[j], S.z[i] - S.z[j]};
        std::copy(v, v + 4, &S.split_pairs[(size_t)id * 4]);
        ++id;
      }
      id = cnt_sup[i];
      for (int slot = 0; slot < NEAR_SLOTS; ++slot) {
        int& f = S.split_sup[(size_t)i * NEAR_SLOTS + slot];
        if (f < 0) continue;
        f = (int)id;
        double dr, dz;
        sup_disp(i, slot, support_pid(S, i, slot), &dr, &dz);
        const double v[4] = {S.r[i], S.z[i], dr, dz};
        std::copy(v, v + 4, &S.split_pairs[(size_t)id * 4]);
        ++id;
      }
    }
  });
}

// ---------------------------------------------------------------- device staging
// Process-wide cache of freed device blocks.  Builds allocate and free
// buffers of several GB (matrices, complex64 copies, residual slices, spectra
// scratch), and mapping or unmapping one costs milliseconds; released blocks
// of at least 64 MiB are kept, per device, up to a cap (32 GiB by default,
// mueller_cache_limit) and handed out again for a request of the same size
// (rounded up to 2 MiB).  Releasing synchronizes the device first, as
// cudaFree does, so no kernel still uses a block when it is reused.  When an
// allocation fails the cache is emptied and the allocation retried.
namespace devcache {
constexpr size_t kMinBlock = (size_t)64 << 20, kRound = (size_t)2 << 20;
std::mutex mu;
std::multimap<std::pair<int, size_t>, void*> blocks;  // (device, bytes) -> block
size_t cached = 0, cap = (size_t)32 << 30;

inline size_t rounded(size_t b) { return (b + kRound - 1) / kRound * kRound; }

void trim() {
  std::lock_guard<std::mutex> capture(lu_capture_mutex());
  std::lock_guard<std::mutex> lk(mu);
  int cur = 0;
  cudaGetDevice(&cur);
  for (auto& e : blocks) {
    cudaSetDevice(e.first.first);
    cudaFree(e.second);
  }
  cudaSetDevice(cur);
  blocks.clear();
  cached = 0;
}

size_t bytes_held() {
  std::lock_guard<std::mutex> lk(mu);
  return cached;
}

cudaError_t alloc(void** p, size_t bytes) {
  const bool big = bytes >= kMinBlock;
  const size_t req = big ? rounded(bytes) : bytes;
  if (big) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    auto it = blocks.find({dev, req});
    if (it != blocks.end()) {
      *p = it->second;
      blocks.erase(it);
      cached -= req;
      return cudaSuccess;
    }
  }
  cudaError_t e = cudaMalloc(p, req);
  if (e != cudaSuccess && bytes_held() > 0) {
    cudaGetLastError();
    trim();
    e = cudaMalloc(p, req);
  }
  return e;
}

void release(void* p, size_t bytes) {
  if (!p) return;
  std::lock_guard<std::mutex> capture(lu_capture_mutex());
  if (bytes >= kMinBlock) {
    const size_t req = rounded(bytes);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceSynchronize();
    std::lock_guard<std::mutex> lk(mu);
    if (cached + req <= cap) {
      blocks.insert({{dev, req}, p});
      cached += req;
      return;
    }
  }
  cudaFree(p);
}
}  // namespace devcache

extern "C" void mueller_cache_trim(void) { devcache::trim(); }

extern "C" size_t mueller_cache_limit(size_t bytes) {
  size_t old;
  {
    std::lock_guard<std::mutex> lk(devcache::mu);
    old = devcache::cap;
    devcache::cap = bytes;
  }
  if (devcache::bytes_held() > bytes) devcache::trim();
  return old;
}

extern "C" size_t mueller_cache_bytes(void) { return devcache::bytes_held(); }

struct DevBuf {
  std::vector<std::pair<void*, size_t>> ptrs;
  ~DevBuf() { for (auto& e : ptrs) devcache::release(e.first, e.second); }
  template <class T>
  cudaError_t alloc(T** p, size_t count) {
    const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    cudaError_t e = devcache::alloc((void**)p, bytes);
    if (e == cudaSuccess) ptrs.push_back({*p, bytes});
    return e;
  }
  size_t size_of(const void* p) const {
    for (const auto& e : ptrs)
      if (e.first == p) return e.second;
    return 0;
  }
  void release(void* p) {  // give one buffer back before the others
    for (size_t k = 0; k < ptrs.size(); ++k)
      if (ptrs[k].first == p) {
        devcache::release(p, ptrs[k].second);
        ptrs.erase(ptrs.begin() + k);
        return;
      }
  }
  template <class T>
  cudaError_t upload(T** p, const std::vector<T>& v, cudaStream_t s) {
    cudaError_t e = alloc(p, v.size());
    if (e != cudaSuccess || v.empty()) return e;
    return cudaMemcpyAsync(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s);
  }
};

static std::vector<double> cos_table(int nphi) {
  std::vector<double> c(nphi);
  for (int t = 0; t < nphi; ++t) c[t] = std::cos(2.0 * M_PI * t / nphi);
  return c;
}
static std::vector<double> s2_table(int nphi) {
  std::vector<double> s(nphi / 2 + 1);
  for (int j = 0; j <= nphi / 2; ++j) {
    double v = std::sin(M_PI * j / nphi);
    s[j] = v * v;
  }
  return s;
}

// The series tables live in constant memory, one copy per device: upload
// them to the current device the first time it is used.
static void ensure_tables() {
  static std::mutex mu;
  static std::vector<char> done;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(mu);
  if (dev < (int)done.size() && done[dev]) return;
  SeriesTables t;
  fill_series_tables(&t);
  upload_series_tables(t);
  if (dev >= (int)done.size()) done.resize(dev + 1, 0);
  done[dev] = 1;
}

// Digits of the cosine matrix b(j, m) = cos(2 pi m j / nl), j = 0..nl/2,
// m < ncols (divided by 2), in the operand layout of the real product: the
// transform over phi of the sampled rows (far-pair bins and support pairs).
// They depend on (nl, ncols) alone, so they are built on the host once per
// device and key and kept until exit (about 21 MB for every grid of the
// ladder up to 512 points at M = 128); the entry is published only after its
// upload has completed, so builds on other streams may use it at once.
static int cos_digits(int nl, int ncols, cudaStream_t s, const __nv_bfloat16** out) {
  static std::mutex mu;
  static std::map<std::tuple<int, int, int>, __nv_bfloat16*> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(mu);
  const auto key = std::make_tuple(dev, nl, ncols);
  auto it = cache.find(key);
  if (it != cache.end()) {
    *out = it->second;
    return MUELLER_OK;
  }
  const int H = nl / 2 + 1, nkt = (H + 15) / 16;
  std::vector<double> cosv((size_t)H * ncols);
  const double two_pi = 6.283185307179586;
  for (int j = 0; j < H; ++j)
    for (int m = 0; m < ncols; ++m) {
      const long long t = ((long long)m * j) % nl;  // the angle reduced exactly
      cosv[(size_t)j * ncols + m] = std::cos(two_pi * (double)t / (double)nl);
    }
  std::vector<__nv_bfloat16> hb(ozaki_real_b_elems(ncols, nkt));
  ozaki_real_b_host(cosv.data(), H, ncols, 2.0, nkt, hb.data());
  __nv_bfloat16* d = nullptr;
  if (cudaMalloc(&d, hb.size() * sizeof(__nv_bfloat16)) != cudaSuccess) {
    cudaGetLastError();
    return fail(MUELLER_ENOMEM, "cosine digit table");
  }
  cudaError_t e = cudaMemcpyAsync(d, hb.data(), hb.size() * sizeof(__nv_bfloat16), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // hb is a host temporary
  if (e != cudaSuccess) {
    cudaFree(d);
    return fail(MUELLER_ECUDA, std::string("cosine digit table: ") + cudaGetErrorString(e));
  }
  cache.emplace(key, d);
  *out = d;
  return MUELLER_OK;
}

// Host-side fault injection for tests (nothing faults on the device): when
// the environment variable MUELLER_FAULT_INJECT names a status word
// ("lu_timeout", "residual_timeout"), the host writes 1 into that device word
// before reading it back, as a bounded device-side wait that gave up would.
static bool fault_injected(const char* what) {
  const char* v = std::getenv("MUELLER_FAULT_INJECT");
  return v && std::strstr(v, what) != nullptr;
}
// Device-to-host reads of status words and small results go through the
// caller's stream (never the legacy default stream, which would join another
// host thread's stream capture).
static void inject_status(int* dev_word, const char* what, cudaStream_t s) {
  if (dev_word && fault_injected(what)) {
    const int one = 1;
    cudaMemcpyAsync(dev_word, &one, sizeof(int), cudaMemcpyHostToDevice, s);
    cudaStreamSynchronize(s);
  }
}

struct Timer {
  cudaEvent_t e[6];
  int n = 0;
  cudaStream_t s;
  explicit Timer(cudaStream_t st) : s(st) { for (auto& x : e) cudaEventCreate(&x); }
  ~Timer() { for (auto& x : e) cudaEventDestroy(x); }
  void mark() { cudaEventRecord(e[n++], s); }
  double ms(int a, int b) { float v = 0; cudaEventElapsedTime(&v, e[a], e[b]); return v; }
};

// Far pairs per chunk of one grid-size bin: digit rows of at most about
// 1.5 GB (18 rows x 16 nkt x 16 bytes per pair), 1024 to 65536 pairs.
static int far_tc_chunk(int nkt) {
  const long long per = 18LL * nkt * 256;
  return (int)std::max<long long>(1024, std::min<long long>(65536, 1500000000LL / per));
}

static size_t far_tc_scratch_bytes(int N, int nphi, int M) {
  const int Ms = M + 2;
  size_t a = 0, y = 0, b = 0, sc = 0;
  for (int nb = 2; nb <= nphi / 8; ++nb) {
    const int nl = 8 * nb, H = nl / 2 + 1, nkt = (H + 15) / 16, ncols = std::min(Ms, nl / 2 + 1);
    const int rp = (far_tc_chunk(nkt) * 2 * NFAM + 127) / 128 * 128;
    a = std::max(a, ozaki_real_a_elems(rp, nkt) * 2);
    y = std::max(y, (size_t)rp * ncols * 8);
    sc = std::max(sc, (size_t)rp * 8);
    b += ozaki_real_b_elems(ncols, nkt) * 2;
  }
  return a + y + sc + b + (size_t)N * N * 6 + 4096;
}

// Far pairs with the transform on the tensor cores (when the largest grid's
// half, n_phi / 2 + 1 samples, fits one exact product), else far_kernel:
// the pairs are binned by their grid (g.nl / 8) on the device, and per bin
// and chunk sampled into digit rows, multiplied by the digits of
// cos(2 pi m j / nl) (modes < min(M + 2, nl / 2 + 1)) and assembled.
struct FarTiming {
  std::vector<cudaEvent_t> ev[3];  // sampling, products, assembly: (start, stop) pairs
  double blocks = 0;
  void mark(int k, cudaStream_t s) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    cudaEventRecord(e, s);
    ev[k].push_back(e);
  }
  // after the stream has synchronised
  void finish(mueller_stats* st) {
    double ms[3] = {0, 0, 0};
    for (int k = 0; k < 3; ++k) {
      for (size_t q = 0; q + 1 < ev[k].size(); q += 2) {
        float v = 0.f;
        cudaEventElapsedTime(&v, ev[k][q], ev[k][q + 1]);
        ms[k] += v;
      }
      for (auto e : ev[k]) cudaEventDestroy(e);
      ev[k].clear();
    }
    if (st) {
      st->ms_far_sample = ms[0]; st->ms_far_product = ms[1]; st->ms_far_assemble = ms[2];
      st->far_blocks = blocks;
    }
  }
  ~FarTiming() { finish(nullptr); }
};

static int far_assembly(const Setup& S, BuildArgs& a, DevBuf& keep_err, int** err_out, FarTiming& ft,
                        cudaStream_t s) {
  const int Ms = S.gp.Ms;
  if (S.gp.H > OZR_KMAX) {
    launch_far_assembly(a, s);
    return MUELLER_OK;
  }
  DevBuf tmp;  // freed (after a device synchronisation) when this returns
  const long long total = (long long)S.N * S.N;
  const int nbins = S.nphi / 8 + 1;
  unsigned short* bin_of = nullptr;
  int *counts = nullptr, *cursor = nullptr, *list = nullptr, *err = nullptr;
  if (tmp.alloc(&bin_of, (size_t)total) != cudaSuccess || tmp.alloc(&counts, (size_t)nbins) != cudaSuccess ||
      tmp.alloc(&cursor, (size_t)nbins) != cudaSuccess || keep_err.alloc(&err, 1) != cudaSuccess)
    return fail(MUELLER_ENOMEM, "far-pair bins");
  CK(cudaMemsetAsync(counts, 0, sizeof(int) * nbins, s));
  CK(cudaMemsetAsync(err, 0, sizeof(int), s));
  launch_far_bins(a, bin_of, counts, s);
  std::vector<int> cnt(nbins), off(nbins + 1, 0);
  CK(cudaMemcpyAsync(cnt.data(), counts, sizeof(int) * nbins, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  for (int b = 0; b < nbins; ++b) off[b + 1] = off[b] + cnt[b];
  *err_out = err;
  if (off[nbins] == 0) return MUELLER_OK;
  if (tmp.alloc(&list, (size_t)off[nbins]) != cudaSuccess) return fail(MUELLER_ENOMEM, "far-pair list");
  CK(cudaMemcpyAsync(cursor, off.data(), sizeof(int) * nbins, cudaMemcpyHostToDevice, s));
  launch_far_scatter(total, bin_of, cursor, list, s);
  // scratch for the largest chunk; the B digits of every bin in use
  size_t amax = 0, ymax = 0, smax = 0;
  std::vector<const __nv_bfloat16*> Bsl(nbins, nullptr);
  for (int b = 2; b < nbins; ++b) {
    if (!cnt[b]) continue;
    const int nl = 8 * b, H = nl / 2 + 1, nkt = (H + 15) / 16, ncols = std::min(Ms, nl / 2 + 1);
    const int cp = std::min(cnt[b], far_tc_chunk(nkt));
    const int rp = (cp * 2 * NFAM + 127) / 128 * 128;
    amax = std::max(amax, ozaki_real_a_elems(rp, nkt));
    ymax = std::max(ymax, (size_t)rp * ncols);
    smax = std::max(smax, (size_t)rp);
    const int rc = cos_digits(nl, ncols, s, &Bsl[b]);
    if (rc != MUELLER_OK) return rc;
  }
  if (cnt[0] || cnt[1]) return fail(MUELLER_EINVAL, "far-pair grid below 16 points");
  __nv_bfloat16* Asl = nullptr;
  double *Ascale = nullptr, *Y = nullptr;
  if (tmp.alloc(&Asl, amax) != cudaSuccess || tmp.alloc(&Ascale, smax) != cudaSuccess ||
      tmp.alloc(&Y, ymax) != cudaSuccess)
    return fail(MUELLER_ENOMEM, "far-pair transform scratch");
  for (int b = 2; b < nbins; ++b) {
    if (!cnt[b]) continue;
    const int nl = 8 * b, H = nl / 2 + 1, nkt = (H + 15) / 16, ncols = std::min(Ms, nl / 2 + 1);
    const int chunk = far_tc_chunk(nkt);
    for (int q0 = 0; q0 < cnt[b]; q0 += chunk) {
      const int c = std::min(chunk, cnt[b] - q0);
      const int rows = c * 2 * NFAM, rp = (rows + 127) / 128 * 128;
      if (rp > rows) {  // the last row tile's padding rows: zero digits and scales
        const int t = rows / 128;
        CK(cudaMemsetAsync(Asl + (size_t)t * nkt * (OZ_S * OZ_RT * OZ_KT), 0,
                           (size_t)nkt * OZ_S * OZ_RT * OZ_KT * sizeof(__nv_bfloat16), s));
        CK(cudaMemsetAsync(Ascale + rows, 0, (size_t)(rp - rows) * sizeof(double), s));
      }
      ft.mark(0, s);
      launch_far_samples(a, list, off[b] + q0, c, Asl, Ascale, nkt, nl, s);
      ft.mark(0, s);
      ft.mark(1, s);
      ozaki_real_gemm(Asl, Ascale, rp, Bsl[b], 2.0, nkt, Y, rp, ncols, err, s);
      ft.mark(1, s);
      ft.mark(2, s);
      launch_far_assemble(a, list, off[b] + q0, c, Y, rp, ncols, nl, s);
      ft.mark(2, s);
      // blocks formed: every pair of the bin assembles modes 0..min(M, m_c + 1), m_c < nl / 2
      ft.blocks += (double)c * std::min(S.M + 1, ncols + 1);
    }
  }
  return MUELLER_OK;
}

// Support pairs per chunk of the tensor-core support transform (its digit and
// product scratch: 18 rows x (16 nkt x 16 + 8 Ms) bytes per pair).
#define SUP_TC_CHUNK 8192

static size_t support_tc_scratch_bytes(int N, int nphi, int M) {
  const int H = nphi / 2 + 1, nkt = (H + 15) / 16, Ms = M + 2;
  const int rows_pad = (SUP_TC_CHUNK * 2 * NFAM + 127) / 128 * 128;
  return ozaki_real_a_elems(rows_pad, nkt) * 2 + (size_t)rows_pad * 8 + (size_t)Ms * rows_pad * 8 +
         ozaki_real_b_elems(Ms, nkt) * 2 + (size_t)N * NEAR_SLOTS * 4 + 64;
}

// Support spectra: on the tensor cores (sampling, digit rows, one real product
// per chunk of pairs, spectra) when the half grid fits one exact product
// (n_phi / 2 + 1 <= OZR_KMAX samples), else the warp-per-pair kernel.
static int support_spectra(const Setup& S, BuildArgs& a, DevBuf& tmp, int** err_out, cudaStream_t s) {
  const int H = S.gp.H, Ms = S.gp.Ms;
  if (H > OZR_KMAX) {
    launch_support_spectra(a, s);
    return MUELLER_OK;
  }
  std::vector<int> list;
  list.reserve((size_t)S.N * (SELF_PTS + 2 * 32));
  for (int i = 0; i < S.N; ++i) {
    const int P = i / P_NODES;
    for (int slot = 0; slot < NEAR_SLOTS; ++slot) {
      if (support_pid(S, i, slot) < 0) continue;
      // the device skips the wrap-around neighbour of a closed curve of one or two panels
      if (slot >= SELF_PTS && S.closed && S.nP <= 2 &&
          ((slot < SELF_PTS + ADJ_PTS && P == 0) || (slot >= SELF_PTS + ADJ_PTS && P == S.nP - 1)))
        continue;
      list.push_back(i * NEAR_SLOTS + slot);
    }
  }
  if (list.empty()) return MUELLER_OK;
  const int nkt = (H + 15) / 16;
  const int rows_pad = (SUP_TC_CHUNK * 2 * NFAM + 127) / 128 * 128;
  int* dlist = nullptr;
  __nv_bfloat16* Asl = nullptr;
  double *Ascale = nullptr, *Y = nullptr;
  int* err = nullptr;
  if (tmp.upload(&dlist, list, s) != cudaSuccess || tmp.alloc(&Asl, ozaki_real_a_elems(rows_pad, nkt)) != cudaSuccess ||
      tmp.alloc(&Ascale, (size_t)rows_pad) != cudaSuccess || tmp.alloc(&Y, (size_t)Ms * rows_pad) != cudaSuccess ||
      tmp.alloc(&err, 1) != cudaSuccess)
    return fail(MUELLER_ENOMEM, "support transform scratch");
  // B: cos(2 pi m j / n_phi), j = 0..n_phi/2 (the samples' weights are in the rows), digits of b / 2
  const __nv_bfloat16* Bsl = nullptr;
  {
    const int rc = cos_digits(S.nphi, Ms, s, &Bsl);
    if (rc != MUELLER_OK) return rc;
  }
  CK(cudaMemsetAsync(err, 0, sizeof(int), s));
  const int total = (int)list.size();
  for (int q0 = 0; q0 < total; q0 += SUP_TC_CHUNK) {
    const int cnt = std::min(SUP_TC_CHUNK, total - q0);
    const int rows = cnt * 2 * NFAM, rp = (rows + 127) / 128 * 128;
    if (rp > rows) {  // the last row tile's padding rows: zero digits and scales
      const int t = rows / 128;
      CK(cudaMemsetAsync(Asl + (size_t)t * nkt * (OZ_S * OZ_RT * OZ_KT), 0,
                         (size_t)nkt * OZ_S * OZ_RT * OZ_KT * sizeof(__nv_bfloat16), s));
      CK(cudaMemsetAsync(Ascale + rows, 0, (size_t)(rp - rows) * sizeof(double), s));
    }
    launch_support_samples(a, dlist, q0, cnt, Asl, Ascale, nkt, s);
    ozaki_real_gemm(Asl, Ascale, rp, Bsl, 2.0, nkt, Y, rp, Ms, err, s);
    launch_support_post(a, dlist, q0, cnt, Y, rp, s);
  }
  *err_out = err;
  return MUELLER_OK;
}

// Assemble modes 0..M into A_dev (column-major per mode, L2-weighted).
static int assemble_core(Setup& S, cd* A_dev, cudaStream_t s, mueller_stats* st, DevBuf& keep,
                         double** d_geo_out) {
  ensure_tables();
  DevBuf tmp;
  BuildArgs a{};
  a.gp = S.gp; a.ap = S.ap; a.N = S.N; a.n_panels = S.nP; a.closed = S.closed;
  double *dr_, *dz_, *drp, *dzp, *dw, *dsw;
  CK(keep.upload(&dr_, S.r, s)); CK(keep.upload(&dz_, S.z, s)); CK(keep.upload(&drp, S.rp, s));
  CK(keep.upload(&dzp, S.zp, s)); CK(keep.upload(&dw, S.w, s)); CK(keep.upload(&dsw, S.sw, s));
  a.geo = NodeGeom{dr_, dz_, drp, dzp, dw, dsw};
  if (d_geo_out) { d_geo_out[0] = dr_; d_geo_out[1] = dz_; d_geo_out[2] = drp; d_geo_out[3] = dzp;
                   d_geo_out[4] = dw; d_geo_out[5] = dsw; }
  double *ssr, *ssz, *ssrp, *sszp, *ssW, *sLs, *sLa, *dcos, *ds2, *dpairs, *dleg, *ssdr, *ssdz;
  int *dsf, *dss;
  CK(tmp.upload(&ssr, S.sr, s)); CK(tmp.upload(&ssz, S.sz, s)); CK(tmp.upload(&ssrp, S.srp, s));
  CK(tmp.upload(&sszp, S.szp, s)); CK(tmp.upload(&ssW, S.sW, s));
  CK(tmp.upload(&ssdr, S.sdr, s)); CK(tmp.upload(&ssdz, S.sdz, s));
  CK(tmp.upload(&sLs, S.Lself, s)); CK(tmp.upload(&sLa, S.Ladj, s));
  int *dadj_rule, *dadj_n;
  CK(tmp.upload(&dadj_rule, S.adj_rule, s)); CK(tmp.upload(&dadj_n, S.adj_n, s));
  CK(tmp.upload(&dcos, cos_table(S.nphi), s)); CK(tmp.upload(&ds2, s2_table(S.nphi), s));
  double *dladC = nullptr, *dladS = nullptr;
  if (S.gp.qmax >= 2) {
    std::vector<double> lc, ls;
    for (int q = 2; q <= S.gp.qmax; ++q) {
      const std::vector<double> c = cos_table(8 * q), t = s2_table(8 * q);
      lc.insert(lc.end(), c.begin(), c.end());
      ls.insert(ls.end(), t.begin(), t.end());
    }
    CK(tmp.upload(&dladC, lc, s)); CK(tmp.upload(&dladS, ls, s));
  }
  CK(tmp.upload(&dsf, S.split_far, s)); CK(tmp.upload(&dss, S.split_sup, s));
  CK(tmp.upload(&dpairs, S.split_pairs, s));
  const long long n_split = (long long)S.split_pairs.size() / 4;
  const int Ms = S.gp.Ms, Mq = S.gp.Mq;
  if (tmp.alloc(&dleg, (size_t)(Mq + 1 + Ms) * n_split) != cudaSuccess)
    return fail(MUELLER_ENOMEM, "Legendre scratch");
  cd* dspec;
  if (tmp.alloc(&dspec, (size_t)S.N * NEAR_SLOTS * NFAM * Ms) != cudaSuccess)
    return fail(MUELLER_ENOMEM, "support spectra scratch");
  a.sup = SupportTable{ssr, ssz, ssrp, sszp, ssW, ssdr, ssdz, sLs, sLa, dadj_rule, dadj_n};
  a.cosT = dcos; a.s2T = ds2; a.ladC = dladC; a.ladS = dladS; a.split_far = dsf; a.split_sup = dss; a.leg = dleg; a.n_split = n_split;
  a.spec_sup = dspec; a.A = A_dev;
  a.lneps = -std::log(S.split_eps);
  a.tq = far_tail_pairs(S.gp);
  a.tailq = nullptr; a.tailij = nullptr;
  if (a.tq) {
    size_t ij = 0;
    const size_t q = far_tail_scratch(a, &ij);
    if (tmp.alloc(&a.tailq, q) != cudaSuccess || tmp.alloc(&a.tailij, ij) != cudaSuccess)
      return fail(MUELLER_ENOMEM, "far-pair tail queue scratch");
  }
  int kc = 8;
  while (kc > 1 && kc * 3 * NFAM * Ms * 16 + NEAR_MAX_PTS * kc * 3 * 8 > 200 * 1024) kc /= 2;
  a.kc = kc;
  Timer T(s);
  T.mark();
  launch_legendre(dpairs, n_split, Mq, Ms, dleg, s);
  T.mark();
  int* far_err = nullptr;
  FarTiming ft;
  {
    const int rc = far_assembly(S, a, tmp, &far_err, ft, s);
    if (rc != MUELLER_OK) return rc;
  }
  T.mark();
  int* sup_err = nullptr;
  {
    const int rc = support_spectra(S, a, tmp, &sup_err, s);
    if (rc != MUELLER_OK) return rc;
  }
  T.mark();
  launch_near_assembly(a, s);
  T.mark();
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  for (int* e : {sup_err, far_err}) {
    if (!e) continue;
    int herr = 0;
    CK(cudaMemcpyAsync(&herr, e, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (herr) return fail(MUELLER_ETIMEOUT, "a device-side wait of the tensor-core kernel transform timed out");
  }
  if (st) ft.finish(st);
  if (st) {
    st->ms_legendre = T.ms(0, 1); st->ms_far = T.ms(1, 2); st->ms_support = T.ms(2, 3); st->ms_near = T.ms(3, 4);
    st->n_phi_used = S.nphi; st->n_split_pairs = n_split; st->n_far_pairs = S.n_far; st->n_support_pairs = S.n_sup;
  }
  return MUELLER_OK;
}

// ---------------------------------------------------------------- context
struct mueller_ctx {
  Setup S;
  DevBuf keep;
  double* geo[6] = {nullptr};  // r, z, rp, zp, w, sw on the device
  cd* A = nullptr;             // FP64 path: factors; mixed path: the weighted matrices [M+1][n][n]
  cf* A32 = nullptr;           // mixed path: complex64 factors
  double* normA = nullptr;     // mixed path: ||A'_m||_inf
  __nv_bfloat16* Asl = nullptr;  // precision 1: digit slices of A' for tensor-core residuals
  double* rowscale = nullptr;
  int npad = 0;
  int* piv = nullptr;
  int* info = nullptr;
  int* tc_err = nullptr;       // set by a timed-out device wait in tensor-core kernels
  int lu_tile = 0;             // column tile of the complex64 update (0: autotuned)
  int launches_pre = 0;        // launches between assembly and LU (norms, conversion, slices)
  size_t bytes = 0;            // device bytes held after the build
  mueller_stats st{};
  // the build's inputs, kept for mueller_ctx_save
  int rec_np = 0, rec_closed = 0, rec_M = 0;
  std::vector<double> rec_r, rec_z, rec_dr, rec_dz;
  mueller_media rec_media{};
  mueller_options rec_opts{};
  // device buffers moved to pinned host memory by mueller_ctx_spill: (field id, bytes, host copy)
  struct HostCopy { int field; size_t bytes; void* host; };
  std::vector<HostCopy> spilled;
  bool is_spilled = false;
  ~mueller_ctx() {
    for (auto& h : spilled) cudaFreeHost(h.host);
  }
};

// The context's device buffers, by a fixed field id (the order of the save file).
static std::vector<void**> ctx_fields(mueller_ctx* c) {
  return {(void**)&c->geo[0], (void**)&c->geo[1], (void**)&c->geo[2], (void**)&c->geo[3], (void**)&c->geo[4],
          (void**)&c->geo[5], (void**)&c->A, (void**)&c->A32, (void**)&c->normA, (void**)&c->Asl,
          (void**)&c->rowscale, (void**)&c->piv, (void**)&c->info, (void**)&c->tc_err};
}

#define SPILLED_CHECK(c) \
  if ((c) && (c)->is_spilled) return fail(MUELLER_EINVAL, "the context's factors are in host memory: call mueller_ctx_restore first")

// Build phases.  prepare: host set-up and the context's allocations;
// assemble: matrices of modes 0..M (plus, mixed path, norms, the complex64
// copy and the digit slices; precision 1 then frees the complex128 matrices);
// factor: the LU of the body's modes (or of a whole wave, mueller_build_many);
// finish: pivot and timeout checks, stats.
static int build_prepare(const mueller_curve* curve, const mueller_media* media, int M, const mueller_options* opts,
                         cudaStream_t s, mueller_ctx** out) {
  *out = nullptr;
  mueller_ctx* c = new mueller_ctx();
  int rc = setup_inputs(curve, media, M, opts, c->S);
  if (rc) { delete c; return rc; }
  if (opts->lu_tile != 0 && opts->lu_tile != 32 && opts->lu_tile != 64 && opts->lu_tile != 128) {
    delete c;
    return fail(MUELLER_EINVAL, "lu_tile must be 0 (autotuned), 32, 64 or 128");
  }
  c->lu_tile = opts->lu_tile;
  c->rec_np = curve->n_panels; c->rec_closed = curve->closed; c->rec_M = M;
  c->rec_r.assign(curve->r, curve->r + c->S.N); c->rec_z.assign(curve->z, curve->z + c->S.N);
  c->rec_dr.assign(curve->dr, curve->dr + c->S.N); c->rec_dz.assign(curve->dz, curve->dz + c->S.N);
  c->rec_media = *media; c->rec_opts = *opts;
  setup_support(curve, c->S);
  setup_pairs(c->S);
  const size_t n = c->S.n;
  const bool mixed = c->S.precision != 0;
  const bool slices = c->S.precision == 1;
  c->npad = (int)((n + OZ_RT - 1) / OZ_RT * OZ_RT);
  const size_t slice_bytes = slices ? ozaki_matrix_slices_elems(c->npad, M + 1) * 2 : 0;
  c->bytes = (size_t)(M + 1) * n * n * (sizeof(cd) + (mixed ? sizeof(cf) : 0)) + slice_bytes;
  size_t freeb = 0, totb = 0;
  cudaMemGetInfo(&freeb, &totb);
  freeb += devcache::bytes_held();  // cached blocks are returned when an allocation needs the room
  if (c->bytes + ((size_t)1 << 30) > freeb) { delete c; return fail(MUELLER_ENOMEM, "factors exceed free device memory"); }
  if (c->keep.alloc(&c->A, (size_t)(M + 1) * n * n) != cudaSuccess ||
      c->keep.alloc(&c->piv, (size_t)(M + 1) * n) != cudaSuccess || c->keep.alloc(&c->info, M + 1) != cudaSuccess ||
      c->keep.alloc(&c->normA, M + 1) != cudaSuccess ||
      (mixed && c->keep.alloc(&c->A32, (size_t)(M + 1) * n * n) != cudaSuccess) ||
      (slices && (c->keep.alloc(&c->Asl, ozaki_matrix_slices_elems(c->npad, M + 1)) != cudaSuccess ||
                  c->keep.alloc(&c->rowscale, (size_t)(M + 1) * c->npad) != cudaSuccess)) ||
      c->keep.alloc(&c->tc_err, 1) != cudaSuccess) {
    delete c;
    return fail(MUELLER_ENOMEM, "factor allocation");
  }
  cudaMemsetAsync(c->tc_err, 0, sizeof(int), s);
  *out = c;
  return MUELLER_OK;
}

static int build_assemble(mueller_ctx* c, cudaStream_t s) {
  const int M = c->S.M;
  const size_t n = c->S.n;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0); cudaEventCreate(&e1);
  cudaEventRecord(e0, s);
  int rc = assemble_core(c->S, c->A, s, &c->st, c->keep, c->geo);
  if (rc) { cudaEventDestroy(e0); cudaEventDestroy(e1); return rc; }
  if (c->S.precision == 0) {  // ||A'_m||_inf for the condition estimate (mueller_cond_estimate)
    mixed_prepare(c->A, (int)n, M + 1, nullptr, c->normA, nullptr, (int)n, s);
    c->launches_pre += 1;
  } else {
    mixed_prepare(c->A, (int)n, M + 1, c->A32, c->normA, c->S.precision == 1 ? c->rowscale : nullptr, c->npad, s);
    c->launches_pre += 1;
    if (c->S.precision == 1) {
      ozaki_slice_matrix(c->A, (int)n, c->npad, M + 1, c->Asl, c->rowscale, s);
      c->launches_pre += 1;
    }
  }
  cudaEventRecord(e1, s);
  cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0); cudaEventDestroy(e1);
  if (err != cudaSuccess) return fail(MUELLER_ECUDA, cudaGetErrorString(err));
  c->st.ms_build = ms;
  if (c->S.precision == 1) {  // the residuals use the slices; the complex128 matrices are no longer needed
    c->keep.release(c->A);
    c->A = nullptr;
    c->bytes -= (size_t)(M + 1) * n * n * sizeof(cd);
  }
  return MUELLER_OK;
}

static int build_finish(mueller_ctx* c, const LuTiming& lt, double ms_lu, int wave_bodies, cudaStream_t s) {
  const int M = c->S.M;
  c->st.ms_lu = ms_lu;
  c->st.ms_build += ms_lu;
  c->st.ms_lu_gemm = lt.gemm_ms; c->st.lu_gemm_flops = lt.gemm_flops; c->st.lu_gemm_launches = lt.gemm_launches;
  c->st.lu_gemm_bytes = lt.gemm_bytes;
  c->st.launches = 4 + c->launches_pre + lt.launches;
  c->st.lu_graph = lt.graph;
  for (int q = 0; q < 3; ++q) c->st.lu_tile_steps[q] = lt.tile_steps[q];
  c->st.lu_wave_bodies = wave_bodies;
  c->st.lu_launches = lt.launches;
  std::vector<int> info(M + 1);
  CK(cudaMemcpyAsync(info.data(), c->info, sizeof(int) * (M + 1), cudaMemcpyDeviceToHost, s));
  int tce = 0;
  inject_status(c->tc_err, "lu_timeout", s);
  CK(cudaMemcpyAsync(&tce, c->tc_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (tce) return fail(MUELLER_ETIMEOUT, "a device-side wait of the tensor-core LU update timed out");
  c->st.singular_mode = -1; c->st.singular_column = -1;
  c->st.kappa_max_mode = -1;
  for (int m = 0; m <= M; ++m)
    if (info[m]) { c->st.singular_mode = m; c->st.singular_column = info[m] - 1; break; }
  c->st.device_bytes = c->bytes;
  return MUELLER_OK;
}

// The (mode) matrices of one body as LU table entries; ws_base: the body's
// complex64 workspace (lu_c64_workspace_bytes(n, M + 1) bytes) or null.
static void lu_items_of(mueller_ctx* c, unsigned char* ws_base, std::vector<LuMat>& items) {
  const int n = c->S.n, M = c->S.M;
  const bool mixed = c->S.precision != 0;
  const size_t wsm = lu_c64_workspace_bytes(n, 1);
  for (int m = 0; m <= M; ++m) {
    void* A = mixed ? (void*)(c->A32 + (size_t)m * n * n) : (void*)(c->A + (size_t)m * n * n);
    items.push_back(LuMat{A, c->piv + (size_t)m * n, c->info + m, ws_base ? ws_base + wsm * m : nullptr, n, 0});
  }
}

extern "C" int mueller_build(const mueller_curve* curve, const mueller_media* media, int M,
                             const mueller_options* opts, void* stream, mueller_ctx** out) {
  g_err.clear();
  if (!out) return fail(MUELLER_EINVAL, "null output pointer");
  *out = nullptr;
  if (!opts) return fail(MUELLER_EINVAL, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  mueller_ctx* c = nullptr;
  int rc = build_prepare(curve, media, M, opts, s, &c);
  if (rc) return rc;
  rc = build_assemble(c, s);
  if (rc) { delete c; return rc; }
  const size_t n = c->S.n;
  const bool mixed = c->S.precision != 0;
  LuTiming lt;
  DevBuf wsb;  // tensor-core LU workspace, freed after the factorisation has completed
  cudaEvent_t e1, e2;
  cudaEventCreate(&e1); cudaEventCreate(&e2);
  cudaEventRecord(e1, s);
  if (mixed) {
    unsigned char* ws = nullptr;
    if (wsb.alloc(&ws, lu_c64_workspace_bytes((int)n, M + 1)) != cudaSuccess) {
      cudaEventDestroy(e1); cudaEventDestroy(e2);
      delete c;
      return fail(MUELLER_ENOMEM, "tensor-core LU workspace");
    }
    lu_factor_batched_c64(c->A32, (int)n, M + 1, c->piv, c->info, s, &lt, c->tc_err, ws, c->lu_tile);
  } else {
    lu_factor_batched(c->A, (int)n, M + 1, c->piv, c->info, s, &lt);
  }
  cudaEventRecord(e2, s);
  cudaError_t err = cudaStreamSynchronize(s);
  float b = 0;
  cudaEventElapsedTime(&b, e1, e2);
  cudaEventDestroy(e1); cudaEventDestroy(e2);
  if (err != cudaSuccess) { delete c; return fail(MUELLER_ECUDA, cudaGetErrorString(err)); }
  rc = build_finish(c, lt, b, 1, s);
  if (rc) { delete c; return rc; }
  *out = c;
  if (c->st.singular_mode >= 0) return fail(MUELLER_ESINGULAR, "exact zero pivot");
  return MUELLER_OK;
}

extern "C" int mueller_build_many(int count, const mueller_curve* curves, const mueller_media* media, const int* M,
                                  const mueller_options* opts, void* stream, mueller_ctx** out) {
  g_err.clear();
  if (!out || !curves || !media || !M || !opts) return fail(MUELLER_EINVAL, "null argument");
  if (count < 1) return fail(MUELLER_EINVAL, "count must be >= 1");
  for (int i = 0; i < count; ++i) out[i] = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<mueller_ctx*> cs(count, nullptr);
  auto drop = [&](int rc) {
    for (auto* c : cs) delete c;
    return rc;
  };
  long long items_total = 0;
  for (int i = 0; i < count; ++i) items_total += (long long)M[i] + 1;
  if (items_total > 65535) return fail(MUELLER_EINVAL, "a wave holds at most 65535 mode matrices");
  for (int i = 0; i < count; ++i) {
    int rc = build_prepare(&curves[i], &media[i], M[i], opts, s, &cs[i]);
    if (rc) return drop(rc);
    rc = build_assemble(cs[i], s);
    if (rc) return drop(rc);
  }
  const bool mixed = opts->precision != 0;
  std::vector<LuMat> items;
  items.reserve((size_t)items_total);
  DevBuf wsb;
  for (int i = 0; i < count; ++i) {
    unsigned char* ws = nullptr;
    if (mixed && wsb.alloc(&ws, lu_c64_workspace_bytes(cs[i]->S.n, M[i] + 1)) != cudaSuccess)
      return drop(fail(MUELLER_ENOMEM, "tensor-core LU workspace"));
    lu_items_of(cs[i], ws, items);
  }
  // one table entry per (body, mode); a body's timeout flag is shared by the wave
  LuTiming lt;
  cudaEvent_t e1, e2;
  cudaEventCreate(&e1); cudaEventCreate(&e2);
  cudaEventRecord(e1, s);
  cudaError_t err = lu_factor_many(items.data(), (int)items.size(), mixed, s, &lt, cs[0]->tc_err,
                                   opts->lu_tile, true);
  cudaEventRecord(e2, s);
  cudaError_t err2 = cudaStreamSynchronize(s);
  float b = 0;
  cudaEventElapsedTime(&b, e1, e2);
  cudaEventDestroy(e1); cudaEventDestroy(e2);
  if (err == cudaSuccess) err = err2;
  if (err != cudaSuccess) return drop(fail(MUELLER_ECUDA, cudaGetErrorString(err)));
  int tce = 0;
  CK(cudaMemcpyAsync(&tce, cs[0]->tc_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  for (int i = 0; i < count; ++i) {
    if (tce) cudaMemcpyAsync(cs[i]->tc_err, cs[0]->tc_err, sizeof(int), cudaMemcpyDeviceToDevice, s);
    int rc = build_finish(cs[i], lt, b, count, s);
    if (rc) return drop(rc);
  }
  bool singular = false;
  for (int i = 0; i < count; ++i) {
    out[i] = cs[i];
    singular = singular || cs[i]->st.singular_mode >= 0;
  }
  if (singular) return fail(MUELLER_ESINGULAR, "exact zero pivot in some body (see its stats)");
  return MUELLER_OK;
}

extern "C" int mueller_assemble(const mueller_curve* curve, const mueller_media* media, int M,
                                const mueller_options* opts, mueller_c128* A_dev, void* stream) {
  g_err.clear();
  if (!A_dev) return fail(MUELLER_EINVAL, "null matrix buffer");
  Setup S;
  int rc = setup_inputs(curve, media, M, opts, S);
  if (rc) return rc;
  setup_support(curve, S);
  setup_pairs(S);
  DevBuf keep;
  return assemble_core(S, (cd*)A_dev, (cudaStream_t)stream, nullptr, keep, nullptr);
}

// Iterative refinement with complex64 factors and FP64 residuals (see mixed.cu).
static int solve_mixed(mueller_ctx* c, const cd* rhs, int nrhs, cd* x, double* backward_err, cudaStream_t s) {
  const int n = c->S.n, M = c->S.M;
  const long long nvec = (long long)(2 * M + 1) * nrhs;
  const bool tcres = c->Asl != nullptr;
  const int ojt = ozaki_job_tile(nrhs), njt = ozaki_job_tiles(nrhs);
  DevBuf tmp;
  cd *bw, *y, *r, *d;
  double* norms;  // [3][nvec]: b', y, r
  __nv_bfloat16* Ysl = nullptr;
  double* colscale = nullptr;
  int* derr = nullptr;
  if (tmp.alloc(&bw, (size_t)nvec * n) || tmp.alloc(&y, (size_t)nvec * n) || tmp.alloc(&r, (size_t)nvec * n) ||
      tmp.alloc(&d, (size_t)nvec * n) || tmp.alloc(&norms, (size_t)3 * nvec) ||
      (tcres && (tmp.alloc(&Ysl, ozaki_vector_slices_elems(c->npad, M + 1, njt, ojt)) ||
                 tmp.alloc(&colscale, (size_t)(M + 1) * njt * ojt) || tmp.alloc(&derr, 1))))
    return fail(MUELLER_ENOMEM, "refinement work vectors");
  if (derr) CK(cudaMemsetAsync(derr, 0, sizeof(int), s));
  double *bn = norms, *yn = norms + nvec, *rn = norms + 2 * nvec;
  std::vector<double> hA(M + 1), hn((size_t)3 * nvec), be((size_t)nvec, 0.0);
  CK(cudaMemcpyAsync(hA.data(), c->normA, sizeof(double) * (M + 1), cudaMemcpyDeviceToHost, s));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0); cudaEventCreate(&e1);
  cudaEventRecord(e0, s);
  mixed_scale(rhs, bw, c->geo[5], n, nvec, bn, s);
  lu_correction_solve_c64(c->A32, c->piv, n, M, bw, d, nrhs, s);
  mixed_update(y, d, n, nvec, true, yn, s);
  int it = 0, launches = 3;
  bool done = false;
  double worst = 0.0;
  std::vector<cudaEvent_t> rev;
  for (; it < c->S.refine_max_iter; ++it) {
    if (tcres) {
      cudaEvent_t a0, a1;
      cudaEventCreate(&a0); cudaEventCreate(&a1);
      cudaEventRecord(a0, s);
      ozaki_residual(c->Asl, c->rowscale, n, c->npad, M, bw, y, r, nrhs, rn, Ysl, colscale, derr, s);
      cudaEventRecord(a1, s);
      rev.push_back(a0); rev.push_back(a1);
      launches += 2;
    } else {
      mixed_residual(c->A, n, M, bw, y, r, nrhs, rn, s);
      launches += 1;
    }
    CK(cudaMemcpyAsync(hn.data(), norms, sizeof(double) * 3 * nvec, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    worst = 0.0;
    for (long long v = 0; v < nvec; ++v) {
      int q = (int)(v / nrhs), m = std::abs(q - M);
      double den = hA[m] * hn[nvec + v] + hn[v];
      be[v] = den > 0 ? hn[2 * nvec + v] / den : 0.0;
      worst = std::max(worst, be[v]);
    }
    if (worst <= c->S.refine_tol) { done = true; break; }
    lu_correction_solve_c64(c->A32, c->piv, n, M, r, d, nrhs, s);
    mixed_update(y, d, n, nvec, false, yn, s);
    launches += 2;
  }
  mixed_unscale(y, x, c->geo[5], n, nvec, s);
  cudaEventRecord(e1, s);
  cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0); cudaEventDestroy(e1);
  if (err != cudaSuccess) return fail(MUELLER_ECUDA, cudaGetErrorString(err));
  c->st.ms_solve = ms;
  c->st.solve_launches = launches + 1;
  c->st.refine_iters = it;
  c->st.ms_residual = 0.0;
  c->st.residual_launches = (int)rev.size() / 2;
  for (size_t q = 0; q + 1 < rev.size(); q += 2) {
    float t = 0.f;
    cudaEventElapsedTime(&t, rev[q], rev[q + 1]);
    c->st.ms_residual += t;
    cudaEventDestroy(rev[q]); cudaEventDestroy(rev[q + 1]);
  }
  // tensor work per residual: 36 digit products x 4 real products of
  // (npad x npad) x (npad x 32 jobs per job tile) per mode, 2 flops per MAC
  c->st.residual_tc_flops = (double)c->st.residual_launches * 144.0 * 2.0 * (double)c->npad * c->npad *
                            ojt * njt * (M + 1);
  c->st.backward_err_max = worst;
  if (backward_err) std::copy(be.begin(), be.end(), backward_err);
  if (derr) {
    int h = 0;
    inject_status(derr, "residual_timeout", s);
    cudaMemcpyAsync(&h, derr, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    if (h) return fail(MUELLER_ETIMEOUT, "a device-side wait of the tensor-core residual timed out");
  }
  if (!done) return fail(MUELLER_ENOCONV, "refinement stopped at refine_max_iter");
  return MUELLER_OK;
}

extern "C" int mueller_solve(mueller_ctx* c, const mueller_c128* rhs_dev, int nrhs, mueller_c128* x_dev,
                             double* backward_err, void* stream) {
  g_err.clear();
  SPILLED_CHECK(c);
  if (!c || !rhs_dev || !x_dev || nrhs < 1) return fail(MUELLER_EINVAL, "invalid solve arguments");
  if ((const void*)rhs_dev == (const void*)x_dev) return fail(MUELLER_EINVAL, "rhs and x must not alias");
  cudaStream_t s = (cudaStream_t)stream;
  if (c->S.precision != 0) return solve_mixed(c, (const cd*)rhs_dev, nrhs, (cd*)x_dev, backward_err, s);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0); cudaEventCreate(&e1);
  cudaEventRecord(e0, s);
  lu_solve_modes(c->A, c->piv, c->S.n, c->S.M, c->geo[5], (const cd*)rhs_dev, (cd*)x_dev, nrhs, s);
  cudaEventRecord(e1, s);
  cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0); cudaEventDestroy(e1);
  if (err != cudaSuccess) return fail(MUELLER_ECUDA, cudaGetErrorString(err));
  c->st.ms_solve = ms;
  c->st.solve_launches = 1;
  if (backward_err)
    for (int q = 0; q < (2 * c->S.M + 1) * nrhs; ++q) backward_err[q] = -1.0;  // not computed on the FP64 path
  return MUELLER_OK;
}

static int n_theta_for(const Setup& S) {  // a multiple of 16: four transform stages in modal_dft
  return (2 * S.M + 2 * (int)std::ceil(cabs(S.k0) * S.rmax) + 64 + 15) / 16 * 16;
}

extern "C" int mueller_rhs_planewave(mueller_ctx* c, const double* dirs, const double* pols, int nrhs,
                                     mueller_c128* rhs_dev, void* stream) {
  g_err.clear();
  SPILLED_CHECK(c);
  if (!c || !dirs || !pols || !rhs_dev || (nrhs < 1 || nrhs > 65535)) return fail(MUELLER_EINVAL, "invalid rhs arguments");
  cudaStream_t s = (cudaStream_t)stream;
  DevBuf tmp;
  double *dd, *dp;
  std::vector<double> vd(dirs, dirs + 3 * nrhs), vp(pols, pols + 3 * nrhs);
  CK(tmp.upload(&dd, vd, s)); CK(tmp.upload(&dp, vp, s));
  FieldGeom g{c->geo[0], c->geo[1], c->geo[2], c->geo[3], c->geo[4], c->S.N};
  launch_rhs_planewave(g, c->S.M, c->S.k0, c->S.omega, c->S.mu0, c->S.sE, c->S.sH, dd, dp, nrhs, n_theta_for(c->S),
                       (cd*)rhs_dev, s);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  return MUELLER_OK;
}

extern "C" int mueller_rhs_fields(mueller_ctx* c, const mueller_c128* EH_dev, int nrhs, int n_theta,
                                  mueller_c128* rhs_dev, void* stream) {
  g_err.clear();
  SPILLED_CHECK(c);
  if (!c || !EH_dev || !rhs_dev || (nrhs < 1 || nrhs > 65535)) return fail(MUELLER_EINVAL, "invalid field-sample arguments");
  if (n_theta < 2 * c->S.M + 2 || n_theta > 2048)
    return fail(MUELLER_EINVAL, "n_theta must lie in [2M+2, 2048]");
  cudaStream_t s = (cudaStream_t)stream;
  FieldGeom g{c->geo[0], c->geo[1], c->geo[2], c->geo[3], c->geo[4], c->S.N};
  launch_rhs_samples(g, c->S.M, c->S.sE, c->S.sH, (const cd*)EH_dev, nrhs, n_theta, (cd*)rhs_dev, s);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  return MUELLER_OK;
}

extern "C" int mueller_eval(mueller_ctx* c, const mueller_c128* x_dev, int nrhs, const double* targets, int ntargets,
                            int region, mueller_c128* out_dev, void* stream) {
  g_err.clear();
  SPILLED_CHECK(c);
  if (!c || !x_dev || !targets || !out_dev || (nrhs < 1 || nrhs > 65535) || ntargets < 1 || (region != 0 && region != 1))
    return fail(MUELLER_EINVAL, "invalid evaluation arguments");
  for (int p = 0; p < 3 * ntargets; ++p)
    if (!std::isfinite(targets[p])) return fail(MUELLER_EINVAL, "non-finite target coordinate");
  const Setup& S = c->S;
  const cd iw = C(0.0, S.omega);
  cd k, cJ, cM, dM, dJ;
  if (region == 0) {  // eq. exteriorfield
    k = S.k0; cJ = -(C(1.0) / (iw * S.eps0)); cM = C(1.0); dM = C(1.0) / (iw * S.mu0); dJ = C(1.0);
  } else if (S.formulation == 0) {  // eq. interiorfield
    k = S.k1; cJ = C(1.0) / (iw * S.eps1); cM = C(-1.0); dM = -(C(1.0) / (iw * S.mu1)); dJ = C(-1.0);
  } else {  // eq. interior_dual
    k = S.k1; cJ = -(C(1.0) / (iw * S.eps0)); cM = S.mu1 / S.mu0; dM = C(1.0) / (iw * S.mu0); dJ = S.eps1 / S.eps0;
  }
  // Quadrature refined for the closest targets: panel P is split into u_P
  // sub-panels of 16 Gauss points (u_P = ceil(1.5 L_P / d_P), 1..16, L_P its
  // length, d_P the smallest meridian-plane distance from a target to its
  // nodes), geometry and currents from the panel's degree-15 interpolants;
  // the azimuthal rule gets 40 r_max / d_min points where that exceeds the
  // default 2M + 2 ceil(|k| r_max) + 64 (at most 8192).
  const Rules& R = rules();
  const int nP = S.nP;
  std::vector<double> tr(ntargets), tz(ntargets);
  for (int p = 0; p < ntargets; ++p) {
    tr[p] = std::hypot(targets[3 * p], targets[3 * p + 1]);
    tz[p] = targets[3 * p + 2];
  }
  std::vector<int> up(nP);
  double dmin_all = 1e300;
  int nsub = 0;
  for (int P = 0; P < nP; ++P) {
    double L = 0.0, d = 1e300;
    for (int q = 0; q < P_NODES; ++q) {
      const int j = P * P_NODES + q;
      L += S.w[j];
      for (int p = 0; p < ntargets; ++p) d = std::min(d, std::hypot(tr[p] - S.r[j], tz[p] - S.z[j]));
    }
    if (!(d > 0.0)) return fail(MUELLER_EINVAL, "a target lies on a node ring");
    dmin_all = std::min(dmin_all, d);
    up[P] = std::max(1, std::min(16, (int)std::ceil(1.5 * L / d)));
    nsub += up[P] * P_NODES;
  }
  std::vector<double> gr(nsub), gz(nsub), grp(nsub), gzp(nsub), gw(nsub), Lm((size_t)nsub * P_NODES);
  std::vector<int> node0(nsub);
  {
    int s_ = 0;
    double Lrow[P_NODES];
    for (int P = 0; P < nP; ++P) {
      const int U = up[P], j0 = P * P_NODES;
      for (int u = 0; u < U; ++u)
        for (int q = 0; q < P_NODES; ++q, ++s_) {
          const double tau = -1.0 + (2.0 * u + 1.0 + R.x16[q]) / U;
          lagrange_row(R, tau, Lrow);
          double r = 0, z = 0, dr = 0, dz = 0;
          for (int k2 = 0; k2 < P_NODES; ++k2) {
            const int j = j0 + k2;
            const double sp = S.w[j] / R.w16[k2];  // |d gamma / d tau| at the node
            r += Lrow[k2] * S.r[j]; z += Lrow[k2] * S.z[j];
            dr += Lrow[k2] * S.rp[j] * sp; dz += Lrow[k2] * S.zp[j] * sp;
            Lm[(size_t)s_ * P_NODES + k2] = Lrow[k2];
          }
          const double sp = std::hypot(dr, dz);
          gr[s_] = r; gz[s_] = z; grp[s_] = dr / sp; gzp[s_] = dz / sp;
          gw[s_] = R.w16[q] / U * sp;
          node0[s_] = j0;
        }
    }
  }
  const int nth_base = 2 * S.M + 2 * (int)std::ceil(cabs(k) * S.rmax) + 64;
  const int nth = std::max(nth_base, std::min(8192, (int)std::ceil(40.0 * S.rmax / dmin_all)));
  cudaStream_t s = (cudaStream_t)stream;
  DevBuf tmp;
  cd *cur, *xs;
  double *X, *dgr, *dgz, *dgrp, *dgzp, *dgw, *dLm;
  int* dn0;
  std::vector<double> vx(targets, targets + 3 * ntargets);
  const long long nvec = (long long)(2 * S.M + 1) * nrhs;
  if (tmp.alloc(&cur, (size_t)nrhs * nsub * nth * 4) != cudaSuccess ||
      tmp.alloc(&xs, (size_t)nvec * 4 * nsub) != cudaSuccess)
    return fail(MUELLER_ENOMEM, "evaluation buffers");
  CK(tmp.upload(&X, vx, s));
  CK(tmp.upload(&dgr, gr, s)); CK(tmp.upload(&dgz, gz, s)); CK(tmp.upload(&dgrp, grp, s));
  CK(tmp.upload(&dgzp, gzp, s)); CK(tmp.upload(&dgw, gw, s)); CK(tmp.upload(&dLm, Lm, s));
  CK(tmp.upload(&dn0, node0, s));
  launch_interp_currents((const cd*)x_dev, 4 * S.N, nsub, dn0, dLm, nvec, xs, s);
  FieldGeom g{dgr, dgz, dgrp, dgzp, dgw, nsub};
  launch_near_field(g, S.M, xs, nrhs, X, ntargets, nth, k, cJ, cM, dM, dJ, cur, (cd*)out_dev, s);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  return MUELLER_OK;
}

extern "C" int mueller_far_field(mueller_ctx* c, const mueller_c128* x_dev, int nrhs, const double* dirs_dev,
                                 int ndir, mueller_c128* E_dev, void* stream) {
  g_err.clear();
  SPILLED_CHECK(c);
  if (!c || !x_dev || !dirs_dev || !E_dev || (nrhs < 1 || nrhs > 65535) || ndir < 1) return fail(MUELLER_EINVAL, "invalid far-field arguments");
  cudaStream_t s = (cudaStream_t)stream;
  int nth = n_theta_for(c->S);
  DevBuf tmp;
  cd* cur;
  if (tmp.alloc(&cur, (size_t)nrhs * c->S.N * nth * 4) != cudaSuccess) return fail(MUELLER_ENOMEM, "ring buffer");
  FieldGeom g{c->geo[0], c->geo[1], c->geo[2], c->geo[3], c->geo[4], c->S.N};
  launch_far_field(g, c->S.M, c->S.k0, c->S.omega, c->S.eps0, (const cd*)x_dev, nrhs, dirs_dev, ndir, nth, cur,
                   (cd*)E_dev, s);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  return MUELLER_OK;
}

extern "C" int mueller_far_field_grid(mueller_ctx* c, const mueller_c128* x_dev, int nrhs, int n_polar,
                                      int n_azim, mueller_c128* E_dev, void* stream) {
  g_err.clear();
  SPILLED_CHECK(c);
  if (!c || !x_dev || !E_dev || (nrhs < 1 || nrhs > 65535) || n_polar < 1 || n_azim < 1 || n_azim > 8192)
    return fail(MUELLER_EINVAL, "invalid far-field grid arguments");
  cudaStream_t s = (cudaStream_t)stream;
  const int M = c->S.M, nth = n_theta_for(c->S);
  DevBuf tmp;
  cd *coef, *F;
  if (tmp.alloc(&coef, (size_t)n_polar * c->S.N * (2 * M + 3)) != cudaSuccess ||
      tmp.alloc(&F, (size_t)nrhs * n_polar * (2 * M + 1) * 3) != cudaSuccess)
    return fail(MUELLER_ENOMEM, "far-field grid buffers");
  FieldGeom g{c->geo[0], c->geo[1], c->geo[2], c->geo[3], c->geo[4], c->S.N};
  launch_far_field_grid(g, M, c->S.k0, c->S.omega, c->S.eps0, (const cd*)x_dev, nrhs, n_polar, n_azim, nth, coef, F,
                        (cd*)E_dev, s);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  return MUELLER_OK;
}

extern "C" int mueller_modal_kernels(const double* pairs_host, long long npairs, mueller_c128 k0, mueller_c128 k1,
                                     int M, int n_phi, double split_eps, mueller_c128* out_dev, void* stream) {
  g_err.clear();
  if (!pairs_host || !out_dev || npairs < 0 || M < 0) return fail(MUELLER_EINVAL, "invalid kernel arguments");
  if (npairs == 0) return MUELLER_OK;
  if (k0.im < 0 || k1.im < 0) return fail(MUELLER_EINVAL, "wavenumbers need Im k >= 0");
  double rmax = 0.0;
  for (long long p = 0; p < npairs; ++p) {
    if (!(pairs_host[4 * p] > 0.0) || !(pairs_host[4 * p + 2] > 0.0)) return fail(MUELLER_EINVAL, "pairs need r > 0");
    double dr = pairs_host[4 * p] - pairs_host[4 * p + 2], dz = pairs_host[4 * p + 1] - pairs_host[4 * p + 3];
    if (dr == 0.0 && dz == 0.0) return fail(MUELLER_EINVAL, "coincident target and source");
    rmax = std::max(rmax, std::max(pairs_host[4 * p], pairs_host[4 * p + 2]));
  }
  ensure_tables();
  double eps = split_eps > 0 ? split_eps : 1e-17;
  int nphi = nphi_needed(M, std::max(cabs(tocd(k0)), cabs(tocd(k1))), rmax, n_phi);
  GreenParams gp{};
  fill_green_params(gp, M, nphi, tocd(k0), tocd(k1));
  if (!green_fits_smem(gp))
    return fail(MUELLER_EINVAL, "n_phi (" + std::to_string(nphi) + ") and M need more shared memory per warp "
                "than a CTA can have");
  std::vector<int> sid(npairs, -1);
  std::vector<double> sp, vp(4 * npairs);
  long long ns = 0;
  const SplitTest split(nphi, M, eps);
  for (long long p = 0; p < npairs; ++p) {
    const double* q = pairs_host + 4 * p;
    double* v = &vp[4 * p];
    v[0] = q[0]; v[1] = q[1]; v[2] = q[0] - q[2]; v[3] = q[1] - q[3];  // target, target - source
    if (split(v[0], v[2], v[3])) {
      sid[p] = (int)ns++;
      sp.insert(sp.end(), v, v + 4);
    }
  }
  cudaStream_t s = (cudaStream_t)stream;
  DevBuf tmp;
  double *dpairs, *dsp, *dleg, *dcos, *ds2;
  int* dsid;
  CK(tmp.upload(&dpairs, vp, s)); CK(tmp.upload(&dsp, sp, s)); CK(tmp.upload(&dsid, sid, s));
  CK(tmp.upload(&dcos, cos_table(nphi), s)); CK(tmp.upload(&ds2, s2_table(nphi), s));
  if (tmp.alloc(&dleg, (size_t)(gp.Mq + 1 + gp.Ms) * ns) != cudaSuccess) return fail(MUELLER_ENOMEM, "scratch");
  launch_legendre(dsp, ns, gp.Mq, gp.Ms, dleg, s);
  launch_pair_spectra(gp, dpairs, dsid, dleg, ns, npairs, dcos, ds2, (cd*)out_dev, s);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  return MUELLER_OK;
}

extern "C" int mueller_lu_batched(mueller_c128* A_dev, int n, int batch, int* piv_dev, int* info_dev, void* stream) {
  g_err.clear();
  if (!A_dev || !piv_dev || !info_dev || n < 1 || batch < 1) return fail(MUELLER_EINVAL, "invalid LU arguments");
  lu_factor_batched((cd*)A_dev, n, batch, piv_dev, info_dev, (cudaStream_t)stream);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  return MUELLER_OK;
}

extern "C" int mueller_lu_batched_c64(mueller_c64* A_dev, int n, int batch, int* piv_dev, int* info_dev,
                                      void* stream) {
  g_err.clear();
  if (!A_dev || !piv_dev || !info_dev || n < 1 || batch < 1) return fail(MUELLER_EINVAL, "invalid LU arguments");
  cudaStream_t s = (cudaStream_t)stream;
  DevBuf tmp;
  int* err = nullptr;
  unsigned char* ws = nullptr;
  if (tmp.alloc(&err, 1) != cudaSuccess || tmp.alloc(&ws, lu_c64_workspace_bytes(n, batch)) != cudaSuccess)
    return fail(MUELLER_ENOMEM, "tensor-core LU workspace");
  CK(cudaMemsetAsync(err, 0, sizeof(int), s));
  lu_factor_batched_c64((cf*)A_dev, n, batch, piv_dev, info_dev, s, nullptr, err, ws);
  CK(cudaGetLastError());
  int herr = 0;
  CK(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (herr) return fail(MUELLER_ETIMEOUT, "a device-side wait of the tensor-core LU update timed out");
  return MUELLER_OK;
}

extern "C" size_t mueller_build_bytes(int N, int M, int precision, size_t* resident) {
  if (N < 1 || M < 0) return 0;
  const size_t n = 4 * (size_t)N, modes = (size_t)M + 1;
  const size_t npad = (n + OZ_RT - 1) / OZ_RT * OZ_RT;
  const size_t A = modes * n * n * sizeof(cd);
  const size_t A32 = precision != 0 ? modes * n * n * sizeof(cf) : 0;
  const size_t sl = precision == 1 ? ozaki_matrix_slices_elems((int)npad, (int)modes) * 2 + modes * npad * 8 : 0;
  const size_t small = modes * n * 4 + modes * 16 + (size_t)N * 64;
  const size_t scratch = (size_t)N * NEAR_SLOTS * NFAM * (size_t)(M + 2) * sizeof(cd) +
                        std::max(support_tc_scratch_bytes(N, 512, M), far_tc_scratch_bytes(N, 512, M));
  if (resident) *resident = (precision == 1 ? 0 : A) + A32 + sl + small;
  return A + A32 + sl + small + scratch;
}

extern "C" size_t mueller_build_many_bytes(int count, const int* N, const int* M, int precision) {
  if (count < 1 || !N || !M) return 0;
  size_t held = 0, extra = 0;
  for (int i = 0; i < count; ++i) {
    size_t res = 0;
    const size_t peak = mueller_build_bytes(N[i], M[i], precision, &res);
    if (peak == 0) return 0;
    // held through the wave's LU: the resident part, plus the complex128
    // matrices where they stay, plus the LU workspace
    const size_t ws = precision != 0 ? lu_c64_workspace_bytes(4 * N[i], M[i] + 1) : 0;
    held += res + ws;
    extra = std::max(extra, peak - res);  // a body's assembly-time surplus, one body at a time
  }
  return held + extra;
}

extern "C" int mueller_lu_tile_table(int* rest_hi, int* count_hi, int* tile, float* ms_per_matrix, int cap) {
  if (cap < 0 || (cap > 0 && (!rest_hi || !count_hi || !tile || !ms_per_matrix))) return -1;
  return lu_tile_table(rest_hi, count_hi, tile, ms_per_matrix, cap);
}

extern "C" size_t mueller_footprint_bytes(int N, int M) {
  return (size_t)16 * (size_t)(4 * N) * (size_t)(4 * N) * (size_t)(2 * M + 1);
}

extern "C" int mueller_stats_get(const mueller_ctx* c, mueller_stats* out) {
  if (!c || !out) return fail(MUELLER_EINVAL, "null argument");
  *out = c->st;
  out->spilled = c->is_spilled ? 1 : 0;
  out->host_bytes = 0;
  for (const auto& h : c->spilled) out->host_bytes += h.bytes;
  if (c->is_spilled) out->device_bytes = 0;
  return MUELLER_OK;
}

// ---------------------------------------------------------------- condition estimate
void launch_cond_estimate(const void* LU, bool c64, const int* piv, int n, int modes, const double* normA, cd* work,
                          double* kappa, cudaStream_t s);

extern "C" int mueller_cond_estimate(mueller_ctx* c, double* kappa, void* stream) {
  g_err.clear();
  if (!c) return fail(MUELLER_EINVAL, "null context");
  SPILLED_CHECK(c);
  cudaStream_t s = (cudaStream_t)stream;
  const int M = c->S.M, n = c->S.n;
  const bool c64 = c->S.precision != 0;
  const void* LU = c64 ? (const void*)c->A32 : (const void*)c->A;
  if (!LU || !c->normA) return fail(MUELLER_EINVAL, "the context holds no factors");
  DevBuf tmp;
  cd* work;
  double* dk;
  if (tmp.alloc(&work, (size_t)(M + 1) * n) != cudaSuccess || tmp.alloc(&dk, M + 1) != cudaSuccess)
    return fail(MUELLER_ENOMEM, "condition-estimate scratch");
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0); cudaEventCreate(&e1);
  cudaEventRecord(e0, s);
  launch_cond_estimate(LU, c64, c->piv, n, M + 1, c->normA, work, dk, s);
  cudaEventRecord(e1, s);
  std::vector<double> hk(M + 1);
  cudaError_t err = cudaMemcpyAsync(hk.data(), dk, sizeof(double) * (M + 1), cudaMemcpyDeviceToHost, s);
  if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0); cudaEventDestroy(e1);
  if (err != cudaSuccess) return fail(MUELLER_ECUDA, cudaGetErrorString(err));
  c->st.kappa_max = -1.0;
  c->st.kappa_max_mode = -1;
  for (int m = 0; m <= M; ++m)
    if (hk[m] > c->st.kappa_max) { c->st.kappa_max = hk[m]; c->st.kappa_max_mode = m; }
  c->st.kappa_mode0 = hk[0];
  c->st.ms_cond = ms;
  if (kappa) std::copy(hk.begin(), hk.end(), kappa);
  return MUELLER_OK;
}

// ---------------------------------------------------------------- host spill and checkpoints
extern "C" int mueller_ctx_spill(mueller_ctx* c, void* stream) {
  g_err.clear();
  if (!c) return fail(MUELLER_EINVAL, "null context");
  if (c->is_spilled) return MUELLER_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const std::vector<void**> fields = ctx_fields(c);
  std::vector<mueller_ctx::HostCopy> copies;
  for (int f = 0; f < (int)fields.size(); ++f) {
    void* p = *fields[f];
    if (!p) continue;
    const size_t bytes = c->keep.size_of(p);
    void* h = nullptr;
    if (cudaMallocHost(&h, bytes) != cudaSuccess) {
      cudaGetLastError();
      cudaStreamSynchronize(s);
      for (auto& x : copies) cudaFreeHost(x.host);
      return fail(MUELLER_ENOMEM, "pinned host memory for the spilled factors");
    }
    copies.push_back({f, bytes, h});
    cudaMemcpyAsync(h, p, bytes, cudaMemcpyDeviceToHost, s);
  }
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    for (auto& x : copies) cudaFreeHost(x.host);
    return fail(MUELLER_ECUDA, cudaGetErrorString(e));
  }
  for (auto& x : copies) {
    c->keep.release(*fields[x.field]);
    *fields[x.field] = nullptr;
  }
  c->spilled = std::move(copies);
  c->is_spilled = true;
  return MUELLER_OK;
}

extern "C" int mueller_ctx_restore(mueller_ctx* c, void* stream) {
  g_err.clear();
  if (!c) return fail(MUELLER_EINVAL, "null context");
  if (!c->is_spilled) return MUELLER_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const std::vector<void**> fields = ctx_fields(c);
  std::vector<void*> got;
  for (const auto& x : c->spilled) {
    char* p = nullptr;
    if (c->keep.alloc(&p, x.bytes) != cudaSuccess) {
      cudaGetLastError();
      cudaStreamSynchronize(s);
      for (void* q : got) c->keep.release(q);
      return fail(MUELLER_ENOMEM, "device memory for the restored factors");
    }
    got.push_back(p);
    cudaMemcpyAsync(p, x.host, x.bytes, cudaMemcpyHostToDevice, s);
  }
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    for (void* q : got) c->keep.release(q);
    return fail(MUELLER_ECUDA, cudaGetErrorString(e));
  }
  for (size_t k = 0; k < c->spilled.size(); ++k) {
    *fields[c->spilled[k].field] = got[k];
    cudaFreeHost(c->spilled[k].host);
  }
  c->spilled.clear();
  c->is_spilled = false;
  return MUELLER_OK;
}

static const char kCkptMagic[8] = {'M', 'U', 'E', 'L', 'C', 'T', 'X', '1'};

extern "C" int mueller_ctx_save(const mueller_ctx* cc, const char* path) {
  g_err.clear();
  if (!cc || !path) return fail(MUELLER_EINVAL, "null argument");
  mueller_ctx* c = const_cast<mueller_ctx*>(cc);  // device pointers are only read
  FILE* f = std::fopen(path, "wb");
  if (!f) return fail(MUELLER_EINVAL, std::string("cannot open ") + path + " for writing");
  bool ok = true;
  auto put = [&](const void* p, size_t b) { if (ok && b && std::fwrite(p, 1, b, f) != b) ok = false; };
  const int32_t version = 1, N = c->S.N;
  put(kCkptMagic, 8); put(&version, 4);
  put(&c->rec_np, 4); put(&c->rec_closed, 4); put(&c->rec_M, 4); put(&N, 4);
  put(c->rec_r.data(), 8 * N); put(c->rec_z.data(), 8 * N); put(c->rec_dr.data(), 8 * N); put(c->rec_dz.data(), 8 * N);
  put(&c->rec_media, sizeof(mueller_media)); put(&c->rec_opts, sizeof(mueller_options));
  put(&c->npad, 4); put(&c->lu_tile, 4); put(&c->launches_pre, 4); put(&c->bytes, 8);
  put(&c->st, sizeof(mueller_stats));
  const std::vector<void**> fields = ctx_fields(c);
  int32_t nf = 0;
  for (int k = 0; k < (int)fields.size(); ++k) nf += (*fields[k] != nullptr) ? 1 : 0;
  nf += (int32_t)c->spilled.size();
  put(&nf, 4);
  std::vector<char> buf;
  for (int k = 0; k < (int)fields.size() && ok; ++k) {
    const void* p = *fields[k];
    const void* host = nullptr;
    uint64_t bytes = 0;
    if (p) {
      bytes = c->keep.size_of(p);
    } else {
      for (const auto& h : c->spilled)
        if (h.field == k) { host = h.host; bytes = h.bytes; }
      if (!host) continue;
    }
    const int32_t id = k;
    put(&id, 4); put(&bytes, 8);
    if (host) { put(host, bytes); continue; }
    const size_t chunk = (size_t)256 << 20;
    buf.resize(std::min<size_t>(chunk, bytes));
    for (size_t o = 0; o < bytes && ok; o += chunk) {
      const size_t b = std::min<size_t>(chunk, bytes - o);
      if (cudaMemcpy(buf.data(), (const char*)p + o, b, cudaMemcpyDeviceToHost) != cudaSuccess) ok = false;
      put(buf.data(), b);
    }
  }
  if (std::fclose(f) != 0) ok = false;
  if (!ok) return fail(MUELLER_EINVAL, std::string("writing ") + path + " failed");
  return MUELLER_OK;
}

extern "C" int mueller_ctx_load(const char* path, void* stream, mueller_ctx** out) {
  g_err.clear();
  if (!path || !out) return fail(MUELLER_EINVAL, "null argument");
  *out = nullptr;
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(MUELLER_EINVAL, std::string("cannot open ") + path);
  bool ok = true;
  auto get = [&](void* p, size_t b) { if (ok && b && std::fread(p, 1, b, f) != b) ok = false; };
  char magic[8] = {0};
  int32_t version = 0, np = 0, closed = 0, M = 0, N = 0;
  get(magic, 8); get(&version, 4);
  if (!ok || std::memcmp(magic, kCkptMagic, 8) != 0 || version != 1) {
    std::fclose(f);
    return fail(MUELLER_EINVAL, std::string(path) + " is not a context checkpoint of this library");
  }
  get(&np, 4); get(&closed, 4); get(&M, 4); get(&N, 4);
  if (!ok || np < 1 || N != 16 * np) { std::fclose(f); return fail(MUELLER_EINVAL, "corrupt checkpoint header"); }
  std::vector<double> r(N), z(N), dr(N), dz(N);
  mueller_media media{};
  mueller_options opts{};
  get(r.data(), 8 * N); get(z.data(), 8 * N); get(dr.data(), 8 * N); get(dz.data(), 8 * N);
  get(&media, sizeof(media)); get(&opts, sizeof(opts));
  if (!ok) { std::fclose(f); return fail(MUELLER_EINVAL, "truncated checkpoint"); }
  mueller_curve cv{np, closed, r.data(), z.data(), dr.data(), dz.data()};
  mueller_ctx* c = new mueller_ctx();
  int rc = setup_inputs(&cv, &media, M, &opts, c->S);
  if (rc) { std::fclose(f); delete c; return rc; }
  c->rec_np = np; c->rec_closed = closed; c->rec_M = M;
  c->rec_r = r; c->rec_z = z; c->rec_dr = dr; c->rec_dz = dz;
  c->rec_media = media; c->rec_opts = opts;
  get(&c->npad, 4); get(&c->lu_tile, 4); get(&c->launches_pre, 4); get(&c->bytes, 8);
  get(&c->st, sizeof(mueller_stats));
  int32_t nf = 0;
  get(&nf, 4);
  const std::vector<void**> fields = ctx_fields(c);
  std::vector<char> buf;
  for (int q = 0; q < nf && ok; ++q) {
    int32_t id = -1;
    uint64_t bytes = 0;
    get(&id, 4); get(&bytes, 8);
    if (!ok || id < 0 || id >= (int)fields.size() || bytes == 0) { ok = false; break; }
    char* p = nullptr;
    if (c->keep.alloc(&p, bytes) != cudaSuccess) {
      std::fclose(f); delete c;
      return fail(MUELLER_ENOMEM, "device memory for the checkpoint's factors");
    }
    *fields[id] = p;
    const size_t chunk = (size_t)256 << 20;
    buf.resize(std::min<size_t>(chunk, bytes));
    for (size_t o = 0; o < bytes && ok; o += chunk) {
      const size_t b = std::min<size_t>(chunk, bytes - o);
      get(buf.data(), b);
      if (ok && cudaMemcpy(p + o, buf.data(), b, cudaMemcpyHostToDevice) != cudaSuccess) ok = false;
    }
  }
  std::fclose(f);
  if (!ok) { delete c; return fail(MUELLER_EINVAL, std::string("reading ") + path + " failed"); }
  (void)stream;
  *out = c;
  return MUELLER_OK;
}

extern "C" void mueller_destroy(mueller_ctx* c) { delete c; }

extern "C" const char* mueller_strerror(int status) {
  switch (status) {
    case MUELLER_OK: return "ok";
    case MUELLER_EINVAL: return "invalid argument";
    case MUELLER_ENOMEM: return "out of memory";
    case MUELLER_ESINGULAR: return "exact zero pivot";
    case MUELLER_ENOCONV: return "iterative refinement did not converge";
    case MUELLER_ETIMEOUT: return "device-side wait timed out";
    case MUELLER_ECUDA: return "CUDA error";
    default: return "unknown status";
  }
}

extern "C" const char* mueller_last_error(void) { return g_err.c_str(); }

void mueller_internal_set_error(const char* msg) { g_err = msg; }
