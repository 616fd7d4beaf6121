// CPU oracle for the QSS source term, its analytic Jacobian and one implicit
// (backward-Euler) step.  TEST INFRASTRUCTURE ONLY: it is called by the test
// suite, by the package's smoke check and by the benchmark's CPU-baseline leg,
// never by the product path.  It shares no code with the CUDA path.
//
// Plain, slow and direct: every quantity is computed from its definition in
// the paper's order, per cell, in the scalar type S.  S = double is the
// reference; S = std::complex<double> gives complex-step derivatives of the
// same code; S = __float128 gives a high-precision rerun.
//
// Paper: Hassanaly et al., "Symbolic construction of the chemical Jacobian of
// quasi-steady state (QSS) chemistries for Exascale computing platforms".
//   rates of progress ............ Section 2.1, Eq. (progRates)
//   net production rates .......... Section 2.1, Eq. (ReacMech)
//   QSS relations ................. Section 2.1, Eq. (QSSi)
//   QSS linear system A C = b ..... Section 2.3, Eq. (full_QSSsystem) -- the
//       printed form is garbled; this file assembles A and b from the exact
//       condition omega_m(C, C_Q) = 0, which is linear in C_Q when every
//       reaction side carries at most one QSS species with coefficient one.
//   resolution order .............. Section 2.3 and Appendix B (Tarjan SCC,
//       condensed order, back substitution, Gaussian elimination with
//       pivoting inside each SCC)
//   state vector phi = (C, T) ..... Section 3.1, Eq. (JacExptr)
//   chain rule through C_QSS ...... Section 3.2, Eq. (JQSS); the derivative of
//       C_QSS follows from the implicit-function theorem applied to
//       A C_QSS + b = 0.
//   temperature row ............... Section 3.2.2 (from the production rates)
// Readings where the paper is silent (units, thermo form, falloff form,
// constant-volume energy equation, QSS species excluded from [M] and from the
// energy sums) are listed in the repository's design notes.
//
// Parity: wdot, C_QSS and J are pinned by closed forms, invariants,
// complex-step and finite differences (tests/test_oracle_*.py).
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <vector>
#include <algorithm>
#include <functional>
#include <quadmath.h>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

typedef std::complex<double> cplx;
typedef __float128 quad;

constexpr double R_GAS = 8.31446261815324;     // J/(mol K)
constexpr double P_STD = 101325.0;             // Pa, standard state of K_c
constexpr double CAL = 4.184;                  // J per cal
constexpr double LN10 = 2.302585092994045684;

// ---- scalar helpers: one set per scalar type ------------------------------
inline double re(double x) { return x; }
inline double re(const cplx& x) { return x.real(); }
inline double re(quad x) { return (double)x; }
inline double sexp(double x) { return std::exp(x); }
inline cplx sexp(const cplx& x) { return std::exp(x); }
inline quad sexp(quad x) { return expq(x); }
inline double slog(double x) { return std::log(x); }
inline cplx slog(const cplx& x) { return std::log(x); }
inline quad slog(quad x) { return logq(x); }
inline double slog10(double x) { return std::log10(x); }
inline cplx slog10(const cplx& x) { return std::log10(x); }
inline quad slog10(quad x) { return log10q(x); }
inline double sabs(double x) { return std::fabs(x); }
inline double sabs(const cplx& x) { return std::fabs(x.real()); }
inline double sabs(quad x) { return (double)fabsq(x); }
// Running error analysis (Wilkinson): v is the value computed in double, e a
// first-order bound on |v - exact| in units of the unit roundoff u = 2^-53,
// assuming every elementary operation (and exp/log/log10) is rounded to
// within u of its exact result.  Evaluating the oracle in this type gives, for
// every output, the rounding-error bound of the oracle's own evaluation order.
struct RE {
  double v, e;
  RE() : v(0.0), e(0.0) {}
  RE(double x) : v(x), e(0.0) {}
  RE(double x, double err) : v(x), e(err) {}
};
inline RE operator+(const RE& a, const RE& b) { double v = a.v + b.v; return RE(v, a.e + b.e + std::fabs(v)); }
inline RE operator-(const RE& a, const RE& b) { double v = a.v - b.v; return RE(v, a.e + b.e + std::fabs(v)); }
inline RE operator-(const RE& a) { return RE(-a.v, a.e); }
inline RE operator*(const RE& a, const RE& b) {
  double v = a.v * b.v;
  return RE(v, std::fabs(a.v) * b.e + a.e * std::fabs(b.v) + std::fabs(v));
}
inline RE operator/(const RE& a, const RE& b) {
  double v = a.v / b.v;
  return RE(v, a.e / std::fabs(b.v) + std::fabs(v) * b.e / std::fabs(b.v) + std::fabs(v));
}
inline RE operator+(const RE& a, double b) { return a + RE(b); }
inline RE operator+(double a, const RE& b) { return RE(a) + b; }
inline RE operator-(const RE& a, double b) { return a - RE(b); }
inline RE operator-(double a, const RE& b) { return RE(a) - b; }
inline RE operator*(const RE& a, double b) { return a * RE(b); }
inline RE operator*(double a, const RE& b) { return RE(a) * b; }
inline RE operator/(const RE& a, double b) { return a / RE(b); }
inline RE operator/(double a, const RE& b) { return RE(a) / b; }
inline double re(const RE& x) { return x.v; }
inline double sabs(const RE& x) { return std::fabs(x.v); }
inline RE sexp(const RE& x) { double v = std::exp(x.v); return RE(v, std::fabs(v) * (x.e + 1.0)); }
inline RE slog(const RE& x) { double v = std::log(x.v); return RE(v, x.e / std::fabs(x.v) + std::fabs(v)); }
inline RE slog10(const RE& x) {
  double v = std::log10(x.v);
  return RE(v, x.e / (std::fabs(x.v) * 2.302585092994045684) + std::fabs(v));
}
inline double errof(double) { return 0.0; }
inline double errof(const RE& x) { return x.e; }

template <class S> S sq(const S& x) { return x * x; }
template <class S> S ipow(const S& x, int n) {
  S r = S(1.0);
  for (int i = 0; i < n; ++i) r = r * x;
  return r;
}

// ---- mechanism ----------------------------------------------------------------
struct Side {
  std::vector<int> sp;   // species index (0..N-1 transported, N..N+Q-1 QSS)
  std::vector<int> nu;   // stoichiometric coefficient
};

struct Reaction {
  Side lhs, rhs;
  bool reversible;            // reverse direction active
  bool forward = true;        // forward direction active (false: reverse-only)
  double A, b, Ea;            // CHEMKIN units (cm-mol-s, cal/mol) as given
  int kind;                   // 0 plain, 1 third body, 2 Troe falloff
  double A0, b0, Ea0;         // low-pressure limit (Troe)
  double alpha, T3, T1, T2;   // Troe parameters (T***, T*, T**)
  std::vector<double> eff;    // [N] collision efficiencies
  // derived
  double lnA_si, Ea_over_R, lnA0_si, Ea0_over_R;
  int qss_l, qss_r;           // QSS index (0..Q-1) on each side, -1 if none
};

struct Mech {
  int N, Q, M;
  std::vector<double> W;                  // [N] kg/mol
  std::vector<double> nasa_lo, nasa_hi;   // [(N+Q)*7]
  std::vector<double> Tmid;               // [N+Q]
  std::vector<Reaction> rx;
  // QSS resolution order: list of groups (QSS indices) in solve order
  std::vector<std::vector<int>> groups;
};

// ---- Tarjan's strongly connected components (Appendix B), recursive -----------
// adj[v] lists the vertices that v needs.  Components come out in an order in
// which every component appears after all the components it needs.
struct TarjanState {
  const std::vector<std::vector<int>>* adj;
  std::vector<int> index, low;
  std::vector<char> on_stack;
  std::vector<int> stack;
  int counter = 0;
  std::vector<std::vector<int>> comps;
  void visit(int v) {
    index[v] = low[v] = counter++;
    stack.push_back(v);
    on_stack[v] = 1;
    for (int w : (*adj)[v]) {
      if (index[w] < 0) {
        visit(w);
        low[v] = std::min(low[v], low[w]);
      } else if (on_stack[w]) {
        low[v] = std::min(low[v], index[w]);
      }
    }
    if (low[v] == index[v]) {
      std::vector<int> comp;
      int w;
      do {
        w = stack.back();
        stack.pop_back();
        on_stack[w] = 0;
        comp.push_back(w);
      } while (w != v);
      std::sort(comp.begin(), comp.end());
      comps.push_back(comp);
    }
  }
};

std::vector<std::vector<int>> tarjan(const std::vector<std::vector<int>>& adj) {
  TarjanState st;
  int n = (int)adj.size();
  st.adj = &adj;
  st.index.assign(n, -1);
  st.low.assign(n, 0);
  st.on_stack.assign(n, 0);
  for (int v = 0; v < n; ++v)
    if (st.index[v] < 0) st.visit(v);
  return st.comps;
}

// ---- thermodynamics (NASA 7-coefficient polynomials) ---------------------------
template <class S>
struct Thermo {
  S cp_R, h_RT, s_R, g_RT, dcpR_dT, dhRT_dT;
};

template <class S>
Thermo<S> nasa(const Mech& m, int s, const S& T, const S& lnT) {
  const double* a = (re(T) < m.Tmid[s]) ? &m.nasa_lo[7 * s] : &m.nasa_hi[7 * s];
  Thermo<S> t;
  S T2 = T * T, T3 = T2 * T, T4 = T3 * T;
  t.cp_R = a[0] + a[1] * T + a[2] * T2 + a[3] * T3 + a[4] * T4;
  t.h_RT = a[0] + a[1] * T / 2.0 + a[2] * T2 / 3.0 + a[3] * T3 / 4.0 + a[4] * T4 / 5.0 + a[5] / T;
  t.s_R = a[0] * lnT + a[1] * T + a[2] * T2 / 2.0 + a[3] * T3 / 3.0 + a[4] * T4 / 4.0 + a[6];
  t.g_RT = t.h_RT - t.s_R;
  t.dcpR_dT = a[1] + 2.0 * a[2] * T + 3.0 * a[3] * T2 + 4.0 * a[4] * T3;
  t.dhRT_dT = (t.cp_R - t.h_RT) / T;
  return t;
}

// ---- per-cell evaluation ------------------------------------------------------
template <class S>
struct CellOut {
  std::vector<S> wdot;   // [N]
  S Tdot;
  std::vector<S> CQ;     // [Q]
  std::vector<S> J;      // [(N+1)*(N+1)] row-major, row i = d(f_i), column j = d/dphi_j
  std::vector<S> A, bvec;  // QSS system, for diagnostics
};

// Gaussian elimination with partial pivoting (first index of max |a| wins).
// a is n x n row-major, rhs is n x nrhs row-major; solution overwrites rhs.
template <class S>
bool gauss_solve(int n, std::vector<S>& a, int nrhs, std::vector<S>& rhs) {
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = sabs(a[k * n + k]);
    for (int i = k + 1; i < n; ++i)
      if (sabs(a[i * n + k]) > best) { best = sabs(a[i * n + k]); p = i; }
    if (best == 0.0) return false;
    if (p != k) {
      for (int j = 0; j < n; ++j) std::swap(a[k * n + j], a[p * n + j]);
      for (int j = 0; j < nrhs; ++j) std::swap(rhs[k * nrhs + j], rhs[p * nrhs + j]);
    }
    for (int i = k + 1; i < n; ++i) {
      S l = a[i * n + k] / a[k * n + k];
      for (int j = k + 1; j < n; ++j) a[i * n + j] = a[i * n + j] - l * a[k * n + j];
      for (int j = 0; j < nrhs; ++j) rhs[i * nrhs + j] = rhs[i * nrhs + j] - l * rhs[k * nrhs + j];
      a[i * n + k] = S(0.0);
    }
  }
  for (int k = n - 1; k >= 0; --k) {
    for (int j = 0; j < nrhs; ++j) {
      S s = rhs[k * nrhs + j];
      for (int i = k + 1; i < n; ++i) s = s - a[k * n + i] * rhs[i * nrhs + j];
      rhs[k * nrhs + j] = s / a[k * n + k];
    }
  }
  return true;
}

// Rate constants of reaction j and their temperature derivative.  kf excludes
// the concentration products; for third-body reactions it excludes [M] too
// (the caller multiplies), for falloff it includes the falloff factor.
template <class S>
struct Rate {
  S kf, kb;            // forward / reverse rate constants
  S dkf_dT, dkb_dT;    // at fixed concentrations (and fixed [M])
  S dkf_dM, dkb_dM;    // d/d[M] (falloff only)
  S M;                 // third-body concentration
};

template <class S>
Rate<S> rate_constants(const Mech& m, const Reaction& r, const S& T, const S& lnT,
                       const std::vector<S>& C, const std::vector<Thermo<S>>& th) {
  Rate<S> out;
  S invT = S(1.0) / T;
  // Arrhenius: k = A T^b exp(-Ea/(R T))
  S kinf = sexp(S(r.lnA_si) + r.b * lnT - r.Ea_over_R * invT);
  S dlnkinf_dT = (r.b + r.Ea_over_R * invT) * invT;
  S Mc = S(0.0);
  if (r.kind != 0)
    for (int k = 0; k < m.N; ++k) Mc = Mc + r.eff[k] * C[k];
  out.M = Mc;
  S kf, dkf_dT, dkf_dM = S(0.0);
  if (r.kind == 0 || r.kind == 1) {
    kf = kinf;
    dkf_dT = kinf * dlnkinf_dT;
  } else {
    // Troe falloff: k = kinf * Pr/(1+Pr) * F,  Pr = k0 [M] / kinf
    S k0 = sexp(S(r.lnA0_si) + r.b0 * lnT - r.Ea0_over_R * invT);
    S dlnk0_dT = (r.b0 + r.Ea0_over_R * invT) * invT;
    S Pr = k0 * Mc / kinf;
    S e3 = sexp(-T / r.T3), e1 = sexp(-T / r.T1), e2 = sexp(-r.T2 * invT);
    S Fcent = (1.0 - r.alpha) * e3 + r.alpha * e1 + e2;
    S dFcent_dT = -(1.0 - r.alpha) * e3 / r.T3 - r.alpha * e1 / r.T1 + e2 * r.T2 * invT * invT;
    S lFc = slog10(Fcent);
    S c = -0.4 - 0.67 * lFc;
    S nn = 0.75 - 1.27 * lFc;
    S lPr = slog10(Pr);
    S x = lPr + c;
    S den = nn - 0.14 * x;
    S f1 = x / den;
    S lF = lFc / (1.0 + f1 * f1);
    S F = sexp(LN10 * lF);
    S g = Pr / (1.0 + Pr);
    kf = kinf * g * F;
    // derivatives: lF(lFc, x(lPr, lFc)) with den depending on lFc and x
    S df1_dx = nn / (den * den);                 // at fixed lFc
    S df1_dnn = -x / (den * den);
    S dlF_df1 = -lFc * 2.0 * f1 / sq(1.0 + f1 * f1);
    S dlF_dlFc_direct = 1.0 / (1.0 + f1 * f1);
    // dx/dlFc = -0.67 ; dnn/dlFc = -1.27
    S dlF_dlFc = dlF_dlFc_direct + dlF_df1 * (df1_dx * (-0.67) + df1_dnn * (-1.27));
    S dlF_dlPr = dlF_df1 * df1_dx;
    S dlFc_dT = dFcent_dT / (Fcent * LN10);
    // d ln k / d ln Pr at fixed T-part: g' = 1/(1+Pr)^2
    // ln kf = ln kinf + ln Pr - ln(1+Pr) + LN10 * lF
    S dlnkf_dlnPr = 1.0 / (1.0 + Pr) + dlF_dlPr;   // LN10 * dlF/dlPr / LN10
    S dlnPr_dT = dlnk0_dT - dlnkinf_dT;
    S dlnkf_dT = dlnkinf_dT + dlnkf_dlnPr * dlnPr_dT + LN10 * dlF_dlFc * dlFc_dT;
    dkf_dT = kf * dlnkf_dT;
    dkf_dM = kf * dlnkf_dlnPr / Mc;   // dlnPr/d[M] = 1/[M]
  }
  out.kf = kf;
  out.dkf_dT = dkf_dT;
  out.dkf_dM = dkf_dM;
  if (r.reversible) {
    // K_c = exp(-sum nu g/RT) * (P_std/(R T))^{sum nu}
    S sum_g = S(0.0), sum_h = S(0.0);
    int dnu = 0;
    for (size_t i = 0; i < r.lhs.sp.size(); ++i) {
      sum_g = sum_g - (double)r.lhs.nu[i] * th[r.lhs.sp[i]].g_RT;
      sum_h = sum_h - (double)r.lhs.nu[i] * th[r.lhs.sp[i]].h_RT;
      dnu -= r.lhs.nu[i];
    }
    for (size_t i = 0; i < r.rhs.sp.size(); ++i) {
      sum_g = sum_g + (double)r.rhs.nu[i] * th[r.rhs.sp[i]].g_RT;
      sum_h = sum_h + (double)r.rhs.nu[i] * th[r.rhs.sp[i]].h_RT;
      dnu += r.rhs.nu[i];
    }
    S lnKc = -sum_g + (double)dnu * slog(S(P_STD / R_GAS) * invT);
    // d lnKc/dT = sum nu h/(R T^2) - dnu/T
    S dlnKc_dT = (sum_h - (double)dnu) * invT;
    S kb = kf * sexp(-lnKc);
    out.kb = kb;
    out.dkb_dT = kb * (dkf_dT / kf - dlnKc_dT);
    if (re(kf) == 0.0) out.dkb_dT = S(0.0);
    out.dkb_dM = (r.kind == 2) ? kb * (dkf_dM / kf) : S(0.0);
    if (r.kind == 2 && re(kf) == 0.0) out.dkb_dM = S(0.0);
  } else {
    out.kb = S(0.0);
    out.dkb_dT = S(0.0);
    out.dkb_dM = S(0.0);
  }
  return out;
}

// Product of concentrations of one side, transported part only, and its
// partial derivatives with respect to each transported participant.
template <class S>
S side_product(const Side& s, int N, const std::vector<S>& C) {
  S p = S(1.0);
  for (size_t i = 0; i < s.sp.size(); ++i)
    if (s.sp[i] < N) p = p * ipow(C[s.sp[i]], s.nu[i]);
  return p;
}
template <class S>
S side_product_deriv(const Side& s, int N, const std::vector<S>& C, int k) {
  // d/dC_k of prod_{transported i} C_i^nu_i
  S p = S(1.0);
  bool found = false;
  for (size_t i = 0; i < s.sp.size(); ++i) {
    if (s.sp[i] >= N) continue;
    if (s.sp[i] == k) {
      found = true;
      p = p * (double)s.nu[i] * ipow(C[k], s.nu[i] - 1);
    } else {
      p = p * ipow(C[s.sp[i]], s.nu[i]);
    }
  }
  return found ? p : S(0.0);
}

// Jacobian variants (Section 3.2.1): JV_EXACT is Eq. (JQSS) in full;
// JV_CONST_QSS drops its second term (C_Q held at the solved values);
// JV_ZERO_QSS drops it and sets C_Q = 0 inside the Jacobian.  t_fd replaces
// the temperature column of the species rows by the central difference of
// Section 3.2.2 with h = 2^(e-20), T in [2^e, 2^(e+1)).  The temperature row
// is always the derivative of Tdot through the species rows in use.
enum { JV_EXACT = 0, JV_CONST_QSS = 1, JV_ZERO_QSS = 2 };

template <class S>
bool eval_cell(const Mech& m, const S* phi /*[N+1] = C, T*/, bool want_jac, bool ordered_qss,
               CellOut<S>& out, int jvar = JV_EXACT, bool t_fd = false,
               const S* cq_given = nullptr) {
  const int N = m.N, Q = m.Q, n = N + 1;
  std::vector<S> C(phi, phi + N);
  S T = phi[N];
  S lnT = slog(T);
  std::vector<Thermo<S>> th(N + Q);
  for (int s = 0; s < N + Q; ++s) th[s] = nasa(m, s, T, lnT);
  std::vector<Rate<S>> rk(m.M);
  for (int j = 0; j < m.M; ++j) {
    rk[j] = rate_constants(m, m.rx[j], T, lnT, C, th);
    if (!m.rx[j].forward) {
      // reverse-only reaction (one-sided linearization): k_b = k_f / K_c is
      // kept, the forward term is removed
      rk[j].kf = S(0.0);
      rk[j].dkf_dT = S(0.0);
      rk[j].dkf_dM = S(0.0);
    }
  }

  // transported-only parts of the forward / reverse terms
  std::vector<S> pf(m.M), pb(m.M), qfp(m.M), qbp(m.M);
  for (int j = 0; j < m.M; ++j) {
    const Reaction& r = m.rx[j];
    pf[j] = side_product(r.lhs, N, C);
    pb[j] = side_product(r.rhs, N, C);
    S kf = rk[j].kf, kb = rk[j].kb;
    if (r.kind == 1) { kf = kf * rk[j].M; kb = kb * rk[j].M; }
    qfp[j] = kf * pf[j];
    qbp[j] = kb * pb[j];
  }
  // ---- QSS linear system: omega_m = sum_n A_mn C_n + b_m = 0 ----------------
  std::vector<S> A(Q * Q, S(0.0)), b(Q, S(0.0));
  for (int j = 0; j < m.M; ++j) {
    const Reaction& r = m.rx[j];
    for (int side = 0; side < 2; ++side) {
      const Side& sd = side == 0 ? r.lhs : r.rhs;
      double sgn = side == 0 ? -1.0 : 1.0;   // nu = nu'' - nu'
      for (size_t i = 0; i < sd.sp.size(); ++i) {
        if (sd.sp[i] < N) continue;
        int mq = sd.sp[i] - N;
        double num = sgn * sd.nu[i];
        // forward term q_f = qfp * C_{qss_l}
        if (r.qss_l >= 0) A[mq * Q + r.qss_l] = A[mq * Q + r.qss_l] + num * qfp[j];
        else b[mq] = b[mq] + num * qfp[j];
        if (r.qss_r >= 0) A[mq * Q + r.qss_r] = A[mq * Q + r.qss_r] - num * qbp[j];
        else b[mq] = b[mq] - num * qbp[j];
      }
    }
  }
  std::vector<S> CQ(Q, S(0.0));
  if (cq_given) {
    // C_Q supplied by the caller: omega(C, T, C_Q) without the QSS solve
    for (int q = 0; q < Q; ++q) CQ[q] = cq_given[q];
  } else if (ordered_qss) {
    // resolution in the condensed order: singletons by division, groups by
    // Gaussian elimination with partial pivoting
    for (const auto& g : m.groups) {
      int gs = (int)g.size();
      std::vector<S> sub(gs * gs), rhs(gs);
      for (int a = 0; a < gs; ++a) {
        S r0 = -b[g[a]];
        for (int nq = 0; nq < Q; ++nq) {
          if (std::find(g.begin(), g.end(), nq) != g.end()) continue;
          r0 = r0 - A[g[a] * Q + nq] * CQ[nq];
        }
        rhs[a] = r0;
        for (int c = 0; c < gs; ++c) sub[a * gs + c] = A[g[a] * Q + g[c]];
      }
      if (gs == 1) {
        if (re(sub[0]) == 0.0) return false;
        CQ[g[0]] = rhs[0] / sub[0];
      } else {
        if (!gauss_solve(gs, sub, 1, rhs)) return false;
        for (int a = 0; a < gs; ++a) CQ[g[a]] = rhs[a];
      }
    }
  } else {
    std::vector<S> a2 = A, rhs(Q);
    for (int i = 0; i < Q; ++i) rhs[i] = -b[i];
    if (Q > 0 && !gauss_solve(Q, a2, 1, rhs)) return false;
    CQ = rhs;
  }
  // ---- progress rates and production rates ----------------------------------
  std::vector<S> qf(m.M), qb(m.M);
  for (int j = 0; j < m.M; ++j) {
    const Reaction& r = m.rx[j];
    qf[j] = qfp[j] * (r.qss_l >= 0 ? CQ[r.qss_l] : S(1.0));
    qb[j] = qbp[j] * (r.qss_r >= 0 ? CQ[r.qss_r] : S(1.0));
  }
  std::vector<S> wdot(N, S(0.0));
  for (int j = 0; j < m.M; ++j) {
    const Reaction& r = m.rx[j];
    S Qj = qf[j] - qb[j];
    for (size_t i = 0; i < r.lhs.sp.size(); ++i)
      if (r.lhs.sp[i] < N) wdot[r.lhs.sp[i]] = wdot[r.lhs.sp[i]] - (double)r.lhs.nu[i] * Qj;
    for (size_t i = 0; i < r.rhs.sp.size(); ++i)
      if (r.rhs.sp[i] < N) wdot[r.rhs.sp[i]] = wdot[r.rhs.sp[i]] + (double)r.rhs.nu[i] * Qj;
  }
  // ---- temperature equation (constant volume) --------------------------------
  S Su = S(0.0), Scv = S(0.0);
  for (int k = 0; k < N; ++k) {
    Su = Su + (th[k].h_RT - 1.0) * wdot[k];
    Scv = Scv + C[k] * (th[k].cp_R - 1.0);
  }
  S Tdot = -T * Su / Scv;
  out.wdot = wdot;
  out.Tdot = Tdot;
  out.CQ = CQ;
  out.A = A;
  out.bvec = b;
  if (!want_jac) return true;

  // ---- Jacobian: J = d omega/d phi |_{C_Q} + d omega/d C_Q * d C_Q/d phi -----
  // Per-reaction partials of Q_j = qf_j - qb_j at fixed C_Q:
  //   dQ_j/dC_k (k < N), dQ_j/dT, and dQ_j/dC_Qm.
  std::vector<S> dQdphi(m.M * n, S(0.0));
  std::vector<S> dQdCQ(m.M * (Q > 0 ? Q : 1), S(0.0));
  for (int j = 0; j < m.M; ++j) {
    const Reaction& r = m.rx[j];
    S cl = r.qss_l >= 0 ? (jvar == JV_ZERO_QSS ? S(0.0) : CQ[r.qss_l]) : S(1.0);
    S cr = r.qss_r >= 0 ? (jvar == JV_ZERO_QSS ? S(0.0) : CQ[r.qss_r]) : S(1.0);
    S kf = rk[j].kf, kb = rk[j].kb;
    S dkf_dT = rk[j].dkf_dT, dkb_dT = rk[j].dkb_dT;
    S Mfac = S(1.0);
    if (r.kind == 1) Mfac = rk[j].M;
    // concentration columns
    for (int k = 0; k < N; ++k) {
      S d = Mfac * (kf * side_product_deriv(r.lhs, N, C, k) * cl -
                    kb * side_product_deriv(r.rhs, N, C, k) * cr);
      if (r.kind == 1) d = d + r.eff[k] * (kf * pf[j] * cl - kb * pb[j] * cr);
      if (r.kind == 2)
        d = d + r.eff[k] * (rk[j].dkf_dM * pf[j] * cl - rk[j].dkb_dM * pb[j] * cr);
      dQdphi[j * n + k] = d;
    }
    dQdphi[j * n + N] = Mfac * (dkf_dT * pf[j] * cl - dkb_dT * pb[j] * cr);
    if (r.qss_l >= 0) dQdCQ[j * Q + r.qss_l] = dQdCQ[j * Q + r.qss_l] + Mfac * kf * pf[j];
    if (r.qss_r >= 0) dQdCQ[j * Q + r.qss_r] = dQdCQ[j * Q + r.qss_r] - Mfac * kb * pb[j];
  }
  // R = d omega_Q / d phi |_{C_Q}  (Q x n);  A = d omega_Q / d C_Q
  std::vector<S> X(Q * n, S(0.0));
  if (Q > 0 && jvar == JV_EXACT) {
    std::vector<S> Rm(Q * n, S(0.0));
    for (int j = 0; j < m.M; ++j) {
      const Reaction& r = m.rx[j];
      for (int side = 0; side < 2; ++side) {
        const Side& sd = side == 0 ? r.lhs : r.rhs;
        double sgn = side == 0 ? -1.0 : 1.0;
        for (size_t i = 0; i < sd.sp.size(); ++i) {
          if (sd.sp[i] < N) continue;
          int mq = sd.sp[i] - N;
          for (int c = 0; c < n; ++c)
            Rm[mq * n + c] = Rm[mq * n + c] + sgn * sd.nu[i] * dQdphi[j * n + c];
        }
      }
    }
    // X = dC_Q/dphi = -A^{-1} R  (dense partial-pivot solve)
    std::vector<S> a2 = A;
    for (int i = 0; i < Q * n; ++i) X[i] = -Rm[i];
    if (!gauss_solve(Q, a2, n, X)) return false;
  }
  std::vector<S> J(n * n, S(0.0));
  for (int j = 0; j < m.M; ++j) {
    const Reaction& r = m.rx[j];
    // total derivative of Q_j with respect to phi
    std::vector<S> dQ(n);
    for (int c = 0; c < n; ++c) {
      S d = dQdphi[j * n + c];
      for (int mq = 0; mq < Q; ++mq) d = d + dQdCQ[j * Q + mq] * X[mq * n + c];
      dQ[c] = d;
    }
    for (int side = 0; side < 2; ++side) {
      const Side& sd = side == 0 ? r.lhs : r.rhs;
      double sgn = side == 0 ? -1.0 : 1.0;
      for (size_t i = 0; i < sd.sp.size(); ++i) {
        if (sd.sp[i] >= N) continue;
        int row = sd.sp[i];
        for (int c = 0; c < n; ++c) J[row * n + c] = J[row * n + c] + sgn * sd.nu[i] * dQ[c];
      }
    }
  }
  if (t_fd) {
    // central difference in T of the full QSS evaluation
    int e2 = 0;
    std::frexp(re(T), &e2);                 // T = f 2^e2, f in [0.5, 1)
    const double h = std::ldexp(1.0, e2 - 21);
    std::vector<S> pp(phi, phi + n), pm(phi, phi + n);
    pp[N] = pp[N] + h;
    pm[N] = pm[N] - h;
    CellOut<S> op, om;
    if (!eval_cell(m, pp.data(), false, ordered_qss, op) ||
        !eval_cell(m, pm.data(), false, ordered_qss, om))
      return false;
    for (int i = 0; i < N; ++i) J[i * n + N] = (op.wdot[i] - om.wdot[i]) / (2.0 * h);
  }
  // temperature row: Tdot = -T Su / Scv
  for (int c = 0; c < N; ++c) {
    S s = S(0.0);
    for (int k = 0; k < N; ++k) s = s + (th[k].h_RT - 1.0) * J[k * n + c];
    J[N * n + c] = -(T * s + Tdot * (th[c].cp_R - 1.0)) / Scv;
  }
  {
    S s1 = S(0.0), s2 = S(0.0), s3 = S(0.0);
    for (int k = 0; k < N; ++k) {
      s1 = s1 + th[k].dhRT_dT * wdot[k] + (th[k].h_RT - 1.0) * J[k * n + N];
      s3 = s3 + C[k] * th[k].dcpR_dT;
    }
    (void)s2;
    J[N * n + N] = -(Su + T * s1 + Tdot * s3) / Scv;
  }
  out.J = J;
  return true;
}

template <class S>
bool cell_phi(const Mech& m, int64_t c, int64_t ld, const double* rho, const double* T,
              const double* Y, std::vector<S>& phi) {
  phi.resize(m.N + 1);
  for (int k = 0; k < m.N; ++k) phi[k] = S(rho[c] * Y[k * ld + c] / m.W[k]);
  phi[m.N] = S(T[c]);
  return true;
}

int nthreads_or_default(int nt) {
#ifdef _OPENMP
  return nt > 0 ? nt : omp_get_max_threads();
#else
  (void)nt;
  return 1;
#endif
}

// Wdot/Jacobian/CQ/status outputs are all optional (nullptr).
template <class S>
int eval_batch(const Mech* m, int64_t ncells, int64_t ld, const double* rho, const double* T,
               const double* Y, double* wdot, double* Tdot, double* jac, double* cq,
               int ordered, int nthreads) {
  const int n = m->N + 1;
  int nfail = 0;
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads_or_default(nthreads)) reduction(+ : nfail)
  for (int64_t c = 0; c < ncells; ++c) {
    std::vector<S> phi;
    cell_phi(*m, c, ld, rho, T, Y, phi);
    CellOut<S> o;
    if (!eval_cell(*m, phi.data(), jac != nullptr, ordered != 0, o)) { nfail++; continue; }
    if (wdot) for (int k = 0; k < m->N; ++k) wdot[k * ld + c] = re(o.wdot[k]);
    if (Tdot) Tdot[c] = re(o.Tdot);
    if (cq) for (int q = 0; q < m->Q; ++q) cq[q * ld + c] = re(o.CQ[q]);
    if (jac) for (int e = 0; e < n * n; ++e) jac[e * ld + c] = re(o.J[e]);
  }
  return nfail;
}

template <class S>
int jac_fd_batch(const Mech* m, int64_t ncells, int64_t ld, const double* rho, const double* T,
                 const double* Y, double dC, double dT, int scheme, double* jac, double* jac_err,
                 int nthreads) {
  const int n = m->N + 1;
  int nfail = 0;
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads_or_default(nthreads)) reduction(+ : nfail)
  for (int64_t c = 0; c < ncells; ++c) {
    std::vector<S> phi;
    cell_phi(*m, c, ld, rho, T, Y, phi);
    CellOut<S> o0;
    if (!eval_cell(*m, phi.data(), false, true, o0)) { nfail++; continue; }
    for (int j = 0; j < n; ++j) {
      double hj = (j < m->N) ? dC : dT;
      std::vector<S> pp = phi, pm = phi;
      pp[j] = pp[j] + hj;
      pm[j] = pm[j] - hj;
      CellOut<S> op, om;
      bool ok = eval_cell(*m, pp.data(), false, true, op);
      if (scheme == 2) ok = ok && eval_cell(*m, pm.data(), false, true, om);
      if (!ok) { nfail++; break; }
      for (int i = 0; i <= m->N; ++i) {
        S fp = i < m->N ? op.wdot[i] : op.Tdot;
        S f0 = i < m->N ? o0.wdot[i] : o0.Tdot;
        S d;
        if (scheme == 2) {
          S fm = i < m->N ? om.wdot[i] : om.Tdot;
          d = (fp - fm) / (2.0 * hj);
        } else {
          d = (fp - f0) / hj;
        }
        jac[(i * n + j) * ld + c] = re(d);
        if (jac_err) jac_err[(i * n + j) * ld + c] = errof(d);
      }
    }
  }
  return nfail;
}

// Newton on G(phi) = phi - phi0 - h f(phi) from phi0, the full J every
// iteration, FP64 partial-pivot solve; stops when the weighted RMS of the
// update is <= 1 (status 0), on an evaluation or solve failure (2) or after
// max_iter iterations (1).  f0 = f(phi0) (the first iterate), f1 = f at the
// last iterate evaluated.
// Newton on G(phi) = phi - cterm - gamma f(phi) from the iterate phi_init
// (backward Euler: cterm = phi_init = phi_n, gamma = h; BDF2: cterm = the
// combination of phi_n and phi_n-1, gamma = beta h).  f0 is f at the first
// iterate, f1 at the last one.
int newton_solve(const Mech& m, const std::vector<double>& phi_init, const std::vector<double>& cterm,
                 double gamma, double rtol, double atol_C, double atol_T, int max_iter,
                 std::vector<double>& phi, std::vector<double>& f0, std::vector<double>& f1,
                 int* iters) {
  const int N = m.N, n = N + 1;
  phi = phi_init;
  int st = 1, it = 0;
  for (it = 1; it <= max_iter; ++it) {
    CellOut<double> o;
    if (!eval_cell(m, phi.data(), true, true, o)) { st = 2; break; }
    std::vector<double> G(n), Mx(n * n);
    for (int i = 0; i < n; ++i) {
      double fi = i < N ? o.wdot[i] : o.Tdot;
      if (it == 1) f0[i] = fi;
      f1[i] = fi;
      G[i] = phi[i] - cterm[i] - gamma * fi;
      for (int j = 0; j < n; ++j) Mx[i * n + j] = (i == j ? 1.0 : 0.0) - gamma * o.J[i * n + j];
    }
    std::vector<double> d(n);
    for (int i = 0; i < n; ++i) d[i] = -G[i];
    if (!gauss_solve(n, Mx, 1, d)) { st = 2; break; }
    double acc = 0.0;
    bool finite = true;
    for (int i = 0; i < n; ++i) {
      phi[i] += d[i];
      double w = rtol * std::fabs(phi[i]) + (i < N ? atol_C : atol_T);
      acc += (d[i] / w) * (d[i] / w);
      if (!std::isfinite(phi[i])) finite = false;
    }
    if (!finite) { st = 2; break; }
    if (std::sqrt(acc / n) <= 1.0) { st = 0; break; }
  }
  if (it > max_iter) it = max_iter;
  *iters = it;
  return st;
}

int be_newton(const Mech& m, const std::vector<double>& phi0, double h_dt, double rtol,
              double atol_C, double atol_T, int max_iter, std::vector<double>& phi,
              std::vector<double>& f0, std::vector<double>& f1, int* iters) {
  return newton_solve(m, phi0, phi0, h_dt, rtol, atol_C, atol_T, max_iter, phi, f0, f1, iters);
}

}  // namespace

// ================================ C ABI ========================================
extern "C" {

// Build a mechanism from flat arrays.  Species 0..N-1 are transported, N..N+Q-1
// QSS.  Reaction j has nl[j] reactants at lsp/lnu[j*4 + i] and nr[j] products
// at rsp/rnu[j*4 + i]; kind[j] is 0 plain, 1 third body, 2 Troe; eff[j*N + k]
// collision efficiencies; arr[j*3 + 0..2] = A, b, Ea; low[j*3 + ..] the
// low-pressure Arrhenius parameters; troe[j*4 + ..] = alpha, T***, T*, T**.
void* oracle_mech_create(int N, int Q, int M, const double* W, const double* nasa_lo,
                         const double* nasa_hi, const double* Tmid, const int* nl, const int* lsp,
                         const int* lnu, const int* nr, const int* rsp, const int* rnu,
                         const int* reversible, const int* kind, const double* arr,
                         const double* low, const double* troe, const double* eff) {
  Mech* m = new Mech;
  m->N = N; m->Q = Q; m->M = M;
  m->W.assign(W, W + N);
  m->nasa_lo.assign(nasa_lo, nasa_lo + 7 * (N + Q));
  m->nasa_hi.assign(nasa_hi, nasa_hi + 7 * (N + Q));
  m->Tmid.assign(Tmid, Tmid + (N + Q));
  m->rx.resize(M);
  for (int j = 0; j < M; ++j) {
    Reaction& r = m->rx[j];
    r.qss_l = r.qss_r = -1;
    int order = 0;
    for (int i = 0; i < nl[j]; ++i) {
      r.lhs.sp.push_back(lsp[j * 4 + i]);
      r.lhs.nu.push_back(lnu[j * 4 + i]);
      order += lnu[j * 4 + i];
      if (lsp[j * 4 + i] >= N) r.qss_l = lsp[j * 4 + i] - N;
    }
    for (int i = 0; i < nr[j]; ++i) {
      r.rhs.sp.push_back(rsp[j * 4 + i]);
      r.rhs.nu.push_back(rnu[j * 4 + i]);
      if (rsp[j * 4 + i] >= N) r.qss_r = rsp[j * 4 + i] - N;
    }
    // reversible[j]: bit 0 = reverse direction active, bit 1 = forward
    // direction removed (reverse-only reaction)
    r.reversible = (reversible[j] & 1) != 0;
    r.forward = (reversible[j] & 2) == 0;
    r.kind = kind[j];
    r.A = arr[j * 3]; r.b = arr[j * 3 + 1]; r.Ea = arr[j * 3 + 2];
    r.A0 = low[j * 3]; r.b0 = low[j * 3 + 1]; r.Ea0 = low[j * 3 + 2];
    r.alpha = troe[j * 4]; r.T3 = troe[j * 4 + 1]; r.T1 = troe[j * 4 + 2]; r.T2 = troe[j * 4 + 3];
    r.eff.assign(eff + (size_t)j * N, eff + (size_t)j * N + N);
    // CHEMKIN cm-mol-s -> SI: (1e-6)^(order-1), order counting [M] for third body
    int ord_inf = order + (r.kind == 1 ? 1 : 0);
    r.lnA_si = std::log(r.A) + (ord_inf - 1) * std::log(1e-6);
    r.Ea_over_R = r.Ea * CAL / R_GAS;
    if (r.kind == 2) {
      r.lnA0_si = std::log(r.A0) + order * std::log(1e-6);
      r.Ea0_over_R = r.Ea0 * CAL / R_GAS;
    } else {
      r.lnA0_si = 0.0;
      r.Ea0_over_R = 0.0;
    }
  }
  // QSS dependency digraph: m needs n when an active direction's rate is
  // proportional to C_n (n its one QSS reactant) and m is a QSS species of
  // the reaction's other side.
  std::vector<std::vector<int>> adj(Q);
  for (int j = 0; j < M; ++j) {
    const Reaction& r = m->rx[j];
    for (int dir = 0; dir < 2; ++dir) {
      if (dir == 0 ? !r.forward : !r.reversible) continue;
      const Side& in = dir == 0 ? r.lhs : r.rhs;
      const Side& other = dir == 0 ? r.rhs : r.lhs;
      int n = -1;
      for (int v : in.sp) if (v >= N) n = v - N;
      if (n < 0) continue;
      for (int v : other.sp)
        if (v >= N && v - N != n) adj[v - N].push_back(n);
    }
  }
  for (auto& a : adj) {
    std::sort(a.begin(), a.end());
    a.erase(std::unique(a.begin(), a.end()), a.end());
  }
  m->groups = tarjan(adj);
  return m;
}

void oracle_mech_free(void* h) { delete (Mech*)h; }

// Number of QSS groups and their layout: group g has sizes[g] members listed
// consecutively in members[] (solve order).
int oracle_qss_groups(void* h, int* sizes, int* members) {
  Mech* m = (Mech*)h;
  int pos = 0;
  for (size_t g = 0; g < m->groups.size(); ++g) {
    if (sizes) sizes[g] = (int)m->groups[g].size();
    for (int v : m->groups[g]) { if (members) members[pos] = v; pos++; }
  }
  return (int)m->groups.size();
}

// Tarjan on an arbitrary digraph given as an edge list (u needs v).
int oracle_tarjan(int nv, int ne, const int* eu, const int* ev, int* comp_of, int* order) {
  std::vector<std::vector<int>> adj(nv);
  for (int e = 0; e < ne; ++e) adj[eu[e]].push_back(ev[e]);
  auto comps = tarjan(adj);
  int pos = 0;
  for (size_t c = 0; c < comps.size(); ++c)
    for (int v : comps[c]) { comp_of[v] = (int)c; order[pos++] = v; }
  return (int)comps.size();
}

// FP64 evaluation.  ordered=1 solves the QSS system in the condensed SCC order,
// ordered=0 with one dense partial-pivot solve (cross-check).
int oracle_eval(void* h, int64_t ncells, int64_t ld, const double* rho, const double* T,
                const double* Y, double* wdot, double* Tdot, double* jac, double* cq,
                int ordered, int nthreads) {
  return eval_batch<double>((Mech*)h, ncells, ld, rho, T, Y, wdot, Tdot, jac, cq, ordered, nthreads);
}

// First-order rounding-error bounds of the FP64 evaluation (units of u = 2^-53)
// for wdot, Tdot and J, computed by running error analysis.
int oracle_eval_errbound(void* h, int64_t ncells, int64_t ld, const double* rho, const double* T,
                         const double* Y, double* wdot_e, double* Tdot_e, double* jac_e,
                         int nthreads) {
  Mech* m = (Mech*)h;
  const int n = m->N + 1;
  int nfail = 0;
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads_or_default(nthreads)) reduction(+ : nfail)
  for (int64_t c = 0; c < ncells; ++c) {
    std::vector<RE> phi;
    cell_phi(*m, c, ld, rho, T, Y, phi);
    CellOut<RE> o;
    if (!eval_cell(*m, phi.data(), jac_e != nullptr, true, o)) { nfail++; continue; }
    if (wdot_e) for (int k = 0; k < m->N; ++k) wdot_e[k * ld + c] = o.wdot[k].e;
    if (Tdot_e) Tdot_e[c] = o.Tdot.e;
    if (jac_e) for (int e = 0; e < n * n; ++e) jac_e[e * ld + c] = o.J[e].e;
  }
  return nfail;
}

// The same evaluation carried out in binary128 and rounded to double.
int oracle_eval_q128(void* h, int64_t ncells, int64_t ld, const double* rho, const double* T,
                     const double* Y, double* wdot, double* Tdot, double* jac, double* cq,
                     int nthreads) {
  return eval_batch<quad>((Mech*)h, ncells, ld, rho, T, Y, wdot, Tdot, jac, cq, 1, nthreads);
}

// Direct evaluation at phi = (C[N], T) given per cell (phi[k*ld + c]) in double.
// Outputs f = (wdot, Tdot) [n][ld] and optionally J [n*n][ld].
int oracle_eval_phi(void* h, int64_t ncells, int64_t ld, const double* phi, double* f,
                    double* jac, int nthreads) {
  Mech* m = (Mech*)h;
  const int n = m->N + 1;
  int nfail = 0;
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads_or_default(nthreads)) reduction(+ : nfail)
  for (int64_t c = 0; c < ncells; ++c) {
    std::vector<double> p(n);
    for (int k = 0; k < n; ++k) p[k] = phi[k * ld + c];
    CellOut<double> o;
    if (!eval_cell(*m, p.data(), jac != nullptr, true, o)) { nfail++; continue; }
    for (int k = 0; k < m->N; ++k) f[k * ld + c] = o.wdot[k];
    f[m->N * ld + c] = o.Tdot;
    if (jac) for (int e = 0; e < n * n; ++e) jac[e * ld + c] = o.J[e];
  }
  return nfail;
}

// Complex-step Jacobian of f = (wdot, Tdot) with respect to phi = (C, T):
// J[:, j] = Im f(phi + i h_j e_j) / h_j,  h_j = hrel * max(|phi_j|, 1).
int oracle_jac_complex_step(void* h, int64_t ncells, int64_t ld, const double* rho,
                            const double* T, const double* Y, double hrel, double* jac,
                            int nthreads) {
  Mech* m = (Mech*)h;
  const int n = m->N + 1;
  int nfail = 0;
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads_or_default(nthreads)) reduction(+ : nfail)
  for (int64_t c = 0; c < ncells; ++c) {
    std::vector<cplx> phi;
    cell_phi(*m, c, ld, rho, T, Y, phi);
    for (int j = 0; j < n; ++j) {
      double hj = hrel * std::max(std::fabs(phi[j].real()), 1.0);
      std::vector<cplx> p = phi;
      p[j] = cplx(p[j].real(), hj);
      CellOut<cplx> o;
      if (!eval_cell(*m, p.data(), false, true, o)) { nfail++; break; }
      for (int i = 0; i < m->N; ++i) jac[(i * n + j) * ld + c] = o.wdot[i].imag() / hj;
      jac[(m->N * n + j) * ld + c] = o.Tdot.imag() / hj;
    }
  }
  return nfail;
}

// Finite-difference Jacobian: central (scheme=2) or one-sided forward (scheme=1)
// with absolute step dC for concentrations and dT for temperature.  With
// jac_err given, the evaluation runs in the running-error type and jac_err
// receives the first-order rounding bound of each entry (units of u).
int oracle_jac_fd(void* h, int64_t ncells, int64_t ld, const double* rho, const double* T,
                  const double* Y, double dC, double dT, int scheme, double* jac, int nthreads) {
  return jac_fd_batch<double>((Mech*)h, ncells, ld, rho, T, Y, dC, dT, scheme, jac, nullptr,
                              nthreads);
}

int oracle_jac_fd_errbound(void* h, int64_t ncells, int64_t ld, const double* rho,
                           const double* T, const double* Y, double dC, double dT, int scheme,
                           double* jac, double* jac_err, int nthreads) {
  return jac_fd_batch<RE>((Mech*)h, ncells, ld, rho, T, Y, dC, dT, scheme, jac, jac_err, nthreads);
}

// A Jacobian variant (jvar: 0 exact, 1 constant-QSS, 2 zero-QSS; t_fd: FD
// temperature column), evaluated in the running-error type: values in jac and
// first-order rounding bounds in jac_err (units of u; may be NULL).  wdot and
// Tdot are the exact source term in every variant.
int oracle_eval_variant(void* h, int64_t ncells, int64_t ld, const double* rho, const double* T,
                        const double* Y, int jvar, int t_fd, double* wdot, double* Tdot,
                        double* jac, double* jac_err, int nthreads) {
  Mech* m = (Mech*)h;
  const int n = m->N + 1;
  if (jvar < JV_EXACT || jvar > JV_ZERO_QSS) return -1;
  int nfail = 0;
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads_or_default(nthreads)) reduction(+ : nfail)
  for (int64_t c = 0; c < ncells; ++c) {
    std::vector<RE> phi;
    cell_phi(*m, c, ld, rho, T, Y, phi);
    CellOut<RE> o;
    if (!eval_cell(*m, phi.data(), true, true, o, jvar, t_fd != 0)) { nfail++; continue; }
    if (wdot) for (int k = 0; k < m->N; ++k) wdot[k * ld + c] = o.wdot[k].v;
    if (Tdot) Tdot[c] = o.Tdot.v;
    for (int e = 0; e < n * n; ++e) {
      jac[e * ld + c] = o.J[e].v;
      if (jac_err) jac_err[e * ld + c] = o.J[e].e;
    }
  }
  return nfail;
}

// Complex-step Jacobian of f = (wdot, Tdot) at FIXED QSS concentrations
// cq[q * ld + c] (no QSS solve): d f(phi; C_Q) / d phi, the definition of the
// constant-QSS (C_Q = solved values) and zero-QSS (C_Q = 0) Jacobians.
int oracle_jac_cs_fixed_cq(void* h, int64_t ncells, int64_t ld, const double* rho,
                           const double* T, const double* Y, const double* cq, double hrel,
                           double* jac, int nthreads) {
  Mech* m = (Mech*)h;
  const int n = m->N + 1;
  int nfail = 0;
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads_or_default(nthreads)) reduction(+ : nfail)
  for (int64_t c = 0; c < ncells; ++c) {
    std::vector<cplx> phi;
    cell_phi(*m, c, ld, rho, T, Y, phi);
    std::vector<cplx> q(m->Q > 0 ? m->Q : 1);
    for (int k = 0; k < m->Q; ++k) q[k] = cplx(cq[k * ld + c], 0.0);
    for (int j = 0; j < n; ++j) {
      double hj = hrel * std::max(std::fabs(phi[j].real()), 1.0);
      std::vector<cplx> p = phi;
      p[j] = cplx(p[j].real(), hj);
      CellOut<cplx> o;
      if (!eval_cell(*m, p.data(), false, true, o, JV_EXACT, false, q.data())) { nfail++; break; }
      for (int i = 0; i < m->N; ++i) jac[(i * n + j) * ld + c] = o.wdot[i].imag() / hj;
      jac[(m->N * n + j) * ld + c] = o.Tdot.imag() / hj;
    }
  }
  return nfail;
}

// QSS diagnostics per cell: the full QSS production rates omega_m recomputed
// reaction by reaction (Eq. ReacMech restricted to QSS rows) at the solved C_Q,
// and the magnitude sum_j |nu_mj| (|q_f| + |q_b|) for scaling.
int oracle_qss_residual(void* h, int64_t ncells, int64_t ld, const double* rho, const double* T,
                        const double* Y, double* resid, double* mag, int nthreads) {
  Mech* m = (Mech*)h;
  const int N = m->N, Q = m->Q;
  int nfail = 0;
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads_or_default(nthreads)) reduction(+ : nfail)
  for (int64_t c = 0; c < ncells; ++c) {
    std::vector<double> phi;
    cell_phi(*m, c, ld, rho, T, Y, phi);
    CellOut<double> o;
    if (!eval_cell(*m, phi.data(), false, true, o)) { nfail++; continue; }
    // full concentration vector
    std::vector<double> Cf(N + Q);
    for (int k = 0; k < N; ++k) Cf[k] = phi[k];
    for (int q = 0; q < Q; ++q) Cf[N + q] = o.CQ[q];
    double Tc = phi[N], lnT = std::log(Tc);
    std::vector<Thermo<double>> th(N + Q);
    for (int s = 0; s < N + Q; ++s) th[s] = nasa(*m, s, Tc, lnT);
    std::vector<double> r(Q, 0.0), mg(Q, 0.0);
    std::vector<double> Cn(phi.begin(), phi.begin() + N);
    for (int j = 0; j < m->M; ++j) {
      const Reaction& rx = m->rx[j];
      Rate<double> k = rate_constants(*m, rx, Tc, lnT, Cn, th);
      double kf = k.kf, kb = k.kb;
      if (rx.kind == 1) { kf *= k.M; kb *= k.M; }
      double qf = kf, qb = kb;
      for (size_t i = 0; i < rx.lhs.sp.size(); ++i) qf *= ipow(Cf[rx.lhs.sp[i]], rx.lhs.nu[i]);
      for (size_t i = 0; i < rx.rhs.sp.size(); ++i) qb *= ipow(Cf[rx.rhs.sp[i]], rx.rhs.nu[i]);
      for (size_t i = 0; i < rx.lhs.sp.size(); ++i)
        if (rx.lhs.sp[i] >= N) {
          r[rx.lhs.sp[i] - N] -= rx.lhs.nu[i] * (qf - qb);
          mg[rx.lhs.sp[i] - N] += rx.lhs.nu[i] * (std::fabs(qf) + std::fabs(qb));
        }
      for (size_t i = 0; i < rx.rhs.sp.size(); ++i)
        if (rx.rhs.sp[i] >= N) {
          r[rx.rhs.sp[i] - N] += rx.rhs.nu[i] * (qf - qb);
          mg[rx.rhs.sp[i] - N] += rx.rhs.nu[i] * (std::fabs(qf) + std::fabs(qb));
        }
    }
    for (int q = 0; q < Q; ++q) { resid[q * ld + c] = r[q]; mag[q * ld + c] = mg[q]; }
  }
  return nfail;
}

// Brute-force QSS concentrations in binary128: Newton iterations on the QSS
// production rates omega_Q(C_Q) = 0 computed reaction by reaction, with a
// Jacobian from one-sided differences in binary128, starting from C_Q = 0.
int oracle_qss_newton_q128(void* h, int64_t ncells, int64_t ld, const double* rho,
                           const double* T, const double* Y, int iters, double* cq,
                           int nthreads) {
  Mech* m = (Mech*)h;
  const int N = m->N, Q = m->Q;
  int nfail = 0;
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads_or_default(nthreads)) reduction(+ : nfail)
  for (int64_t c = 0; c < ncells; ++c) {
    std::vector<quad> C(N);
    for (int k = 0; k < N; ++k) C[k] = (quad)rho[c] * (quad)Y[k * ld + c] / (quad)m->W[k];
    quad Tc = T[c], lnT = logq(Tc);
    std::vector<Thermo<quad>> th(N + Q);
    for (int s = 0; s < N + Q; ++s) th[s] = nasa(*m, s, Tc, lnT);
    std::vector<quad> kf(m->M), kb(m->M);
    for (int j = 0; j < m->M; ++j) {
      Rate<quad> k = rate_constants(*m, m->rx[j], Tc, lnT, C, th);
      kf[j] = k.kf; kb[j] = k.kb;
      if (m->rx[j].kind == 1) { kf[j] *= k.M; kb[j] *= k.M; }
    }
    auto omegaQ = [&](const std::vector<quad>& cqv, std::vector<quad>& out) {
      out.assign(Q, (quad)0);
      for (int j = 0; j < m->M; ++j) {
        const Reaction& rx = m->rx[j];
        quad qf = kf[j], qb = kb[j];
        for (size_t i = 0; i < rx.lhs.sp.size(); ++i) {
          int s = rx.lhs.sp[i];
          qf *= ipow(s < N ? C[s] : cqv[s - N], rx.lhs.nu[i]);
        }
        for (size_t i = 0; i < rx.rhs.sp.size(); ++i) {
          int s = rx.rhs.sp[i];
          qb *= ipow(s < N ? C[s] : cqv[s - N], rx.rhs.nu[i]);
        }
        for (size_t i = 0; i < rx.lhs.sp.size(); ++i)
          if (rx.lhs.sp[i] >= N) out[rx.lhs.sp[i] - N] -= rx.lhs.nu[i] * (qf - qb);
        for (size_t i = 0; i < rx.rhs.sp.size(); ++i)
          if (rx.rhs.sp[i] >= N) out[rx.rhs.sp[i] - N] += rx.rhs.nu[i] * (qf - qb);
      }
    };
    std::vector<quad> x(Q, (quad)0), f0, f1;
    bool ok = true;
    for (int it = 0; it < iters && ok; ++it) {
      omegaQ(x, f0);
      std::vector<quad> Jm(Q * Q);
      for (int q = 0; q < Q; ++q) {
        std::vector<quad> xp = x;
        quad hq = (x[q] != 0 ? fabsq(x[q]) : (quad)1) * (quad)1e-20;
        xp[q] += hq;
        omegaQ(xp, f1);
        for (int i = 0; i < Q; ++i) Jm[i * Q + q] = (f1[i] - f0[i]) / hq;
      }
      std::vector<quad> rhs(Q);
      for (int i = 0; i < Q; ++i) rhs[i] = -f0[i];
      ok = gauss_solve(Q, Jm, 1, rhs);
      for (int i = 0; i < Q; ++i) x[i] += rhs[i];
    }
    if (!ok) { nfail++; continue; }
    for (int q = 0; q < Q; ++q) cq[q * ld + c] = (double)x[q];
  }
  return nfail;
}

// One backward-Euler step at constant volume: Newton on
//   G(phi) = phi - phi0 - dt f(phi) = 0,  G' = I - dt J,
// full J re-evaluated every iteration, partial-pivot LU in double.  Stops when
// the weighted RMS norm of the Newton update, weights 1/(rtol|phi_i| + atol_i)
// (atol_C for concentrations, atol_T for temperature), is <= 1, or after
// max_iter iterations.  T and Y are updated in place (rho fixed); iters and
// status (0 converged, 1 not converged, 2 evaluation failure) per cell.
int oracle_be_step(void* h, int64_t ncells, int64_t ld, const double* dt, int dt_stride,
                   const double* rho, double* T, double* Y, double rtol, double atol_C,
                   double atol_T, int max_iter, int* iters, int* status, int nthreads) {
  Mech* m = (Mech*)h;
  const int N = m->N, n = N + 1;
  int nbad = 0;
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads_or_default(nthreads)) reduction(+ : nbad)
  for (int64_t c = 0; c < ncells; ++c) {
    double h_dt = dt[dt_stride ? c : 0];
    std::vector<double> phi0;
    cell_phi(*m, c, ld, rho, T, Y, phi0);
    std::vector<double> phi, f0(n), f1(n);
    int it = 0;
    int st = be_newton(*m, phi0, h_dt, rtol, atol_C, atol_T, max_iter, phi, f0, f1, &it);
    if (iters) iters[c] = it;
    if (status) status[c] = st;
    if (st != 0) nbad++;
    T[c] = phi[N];
    for (int k = 0; k < N; ++k) Y[k * ld + c] = phi[k] * m->W[k] / rho[c];
  }
  return nbad;
}

// Integration over dt_total by substeps with local error control (each cell
// on its own), of order 1 (backward Euler) or 2 (variable-step BDF2 after a
// first backward-Euler substep).  A substep of size h from phi_n is the
// Newton solve above:
//   order 1:  phi - phi_n - h f(phi) = 0;
//   BDF2 (previous accepted substep h_p, w = h / h_p):
//     phi - a1 phi_n - a2 phi_n-1 - beta h f(phi) = 0,
//     a1 = (1+w)^2/(1+2w), a2 = -w^2/(1+2w), beta = (1+w)/(1+2w)
//   (the quadratic through t_n-1, t_n, t_n+1 with slope f at t_n+1).
// Local error estimates from f at the first iterate (f_n) and the last (f_n+1):
//   order 1:  e = h/2 (f_n+1 - f_n)                       (h^2/2 times phi'');
//   BDF2:     e = h (1+w)/(3(1+2w)) ((f_n+1 - f_n) - w (f_n - f_n-1)),
// the formula's truncation error (1+w)^2/(6w(1+2w)) h^3 d3phi/dt3 with the
// third derivative from the second divided difference of f over t_n-1, t_n,
// t_n+1.  err = sqrt(mean((e_i / w_i)^2)), w_i = rtol |phi_i,new| + atol_i.
// Accepted when err <= 1: next h = h min(g_max, max(0.2, 0.9 err^(-1/(p+1))))
// (p the substep's order; g_max = 4 for order 1, 2 for order 2, which keeps
// the step ratio inside BDF2's zero-stability bound 1 + sqrt 2), capped by
// what remains; rejected: h max(0.2, min(0.9, 0.9 err^(-1/(p+1)))); Newton
// failure: h/4.  The interval is done when the remainder is <= 1e-12
// dt_total; a cell fails (status 2) when h < h_min dt_total, and stops with
// status 1 after max_rounds attempts.
int oracle_integrate(void* h, int64_t ncells, int64_t ld, const double* dt_total, int dt_stride,
                     const double* rho, double* T, double* Y, double rtol, double atol_C,
                     double atol_T, double h0, double h_min, int max_rounds, double n_rtol,
                     double n_atol_C, double n_atol_T, int max_iter, int order, int* nsteps,
                     int* status, int nthreads) {
  Mech* m = (Mech*)h;
  const int N = m->N, n = N + 1;
  if (order != 1 && order != 2) return -1;
  const double g_max = order == 2 ? 2.0 : 4.0;
  int nbad = 0;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads_or_default(nthreads)) reduction(+ : nbad)
  for (int64_t c = 0; c < ncells; ++c) {
    const double D = dt_total[dt_stride ? c : 0];
    std::vector<double> phi;
    cell_phi(*m, c, ld, rho, T, Y, phi);
    double t = 0.0, hs = std::min(h0 > 0.0 ? h0 : 0.01 * D, D);
    std::vector<double> phi_prev(n), f_prev(n), cterm(n);
    double h_prev = 0.0;   // 0: no previous substep (the first substep is backward Euler)
    int st = 1, ns = 0;
    for (int round = 0; round < max_rounds; ++round) {
      const bool bdf2 = order == 2 && h_prev > 0.0;
      const double w = bdf2 ? hs / h_prev : 0.0;
      double gamma = hs;
      if (bdf2) {
        const double a1 = (1.0 + w) * (1.0 + w) / (1.0 + 2.0 * w), a2 = -w * w / (1.0 + 2.0 * w);
        for (int i = 0; i < n; ++i) cterm[i] = a1 * phi[i] + a2 * phi_prev[i];
        gamma = (1.0 + w) / (1.0 + 2.0 * w) * hs;
      } else {
        cterm = phi;
      }
      std::vector<double> pn, f0(n), f1(n);
      int it = 0;
      const int ok = newton_solve(*m, phi, cterm, gamma, n_rtol, n_atol_C, n_atol_T, max_iter, pn, f0,
                                  f1, &it);
      if (ok != 0) {
        hs *= 0.25;
      } else {
        double e2 = 0.0;
        const double ce = bdf2 ? hs * (1.0 + w) / (3.0 * (1.0 + 2.0 * w)) : 0.5 * hs;
        for (int i = 0; i < n; ++i) {
          const double e = bdf2 ? ce * ((f1[i] - f0[i]) - w * (f0[i] - f_prev[i])) : ce * (f1[i] - f0[i]);
          const double wt = rtol * std::fabs(pn[i]) + (i < N ? atol_C : atol_T);
          e2 += (e / wt) * (e / wt);
        }
        const double err = std::sqrt(e2 / n);
        // 0.9 err^(-1/(p+1)) for the substep's order p
        const double gr = err > 0.0 ? (bdf2 ? 0.9 / std::cbrt(err) : 0.9 / std::sqrt(err)) : 0.0;
        if (err <= 1.0) {
          if (order == 2) {
            phi_prev = phi;
            f_prev = f0;
            h_prev = hs;
          }
          phi = pn;
          t += hs;
          ns++;
          const double rem = D - t;
          if (rem <= 1e-12 * D) { st = 0; break; }
          const double g = err > 0.0 ? gr : g_max;
          hs = std::min(hs * std::min(g_max, std::max(0.2, g)), rem);
        } else {
          const double g = err > 0.0 ? gr : 0.25;
          hs = hs * (g == g ? std::min(0.9, std::max(0.2, g)) : 0.25);
        }
      }
      if (hs < h_min * D) { st = 2; break; }
    }
    if (nsteps) nsteps[c] = ns;
    if (status) status[c] = st;
    if (st != 0) nbad++;
    T[c] = phi[N];
    for (int k = 0; k < N; ++k) Y[k * ld + c] = phi[k] * m->W[k] / rho[c];
  }
  return nbad;
}

}  // extern "C"
