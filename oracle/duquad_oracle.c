/*
 * duquad_oracle.c -- plain, slow, FP64 CPU oracle of the inexact (augmented)
 * dual first-order method DFOM with inner Algorithm FOM (Necoara & Patrascu,
 * "DuQuad: an inexact (augmented) dual first order algorithm for quadratic
 * programming", arXiv 1504.05708).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: it exists so that the tests, the smoke check and the CPU
 * baseline leg of the benchmark have an independent, obviously correct
 * reference.  It shares no code, header, table or helper with the CUDA path.
 *
 * Conventions (all FP64, IEEE round-to-nearest, no blocking, no fusion):
 *   problem  (eq. original_primal, Sec. 2):
 *       min_{u in U} F(u) = 1/2 u'Qu + q'u   s.t.  Gu + g in K,
 *       U = [lb, ub] (box), K = R^p_- (cone 0, inequalities) or {0} (cone 1).
 *   Q is n x n row-major (symmetric), G is p x n row-major.
 *   rho >= 0 is the augmentation (Case 1: rho = 0, Case 2: rho > 0).
 *
 * Every function cites the passage of the paper it writes out.  Where the
 * paper leaves a choice open the reading taken is named at the place it is
 * used (inner solver variant, stopping certificate, averaging base).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_CONE_INEQ 0 /* K = R^p_-            */
#define ORC_CONE_EQ 1   /* K = {0}              */

#define ORC_DGM 0
#define ORC_DFGM 1
#define ORC_ADGM 2
#define ORC_ADFGM 3

#define ORC_INNER_AUTO 0     /* FGM_sigma if sigma > 0, else FGM */
#define ORC_INNER_GM 1
#define ORC_INNER_FGM 2
#define ORC_INNER_FGMSIGMA 3

#define ORC_TRACE_COLS 12

typedef struct {
  int n, p, cone;
  const double *Q, *q, *G, *g, *lb, *ub;
} orc_qp;

typedef struct {
  int alg;             /* ORC_DGM .. ORC_ADFGM                              */
  double rho;          /* augmentation; must be 0 for DGM/DFGM              */
  double LL;           /* Lipschitz constant of grad_u L_rho(., mu)         */
  double sigma;        /* strong-convexity lower bound of L_rho(., mu)      */
  double Ld;           /* Lipschitz constant of grad d_rho (eq. Ld)         */
  int kd_literal;      /* 1: K_d = R^p when sigma == 0 (paper's literal K_d) */
  int inner_variant;   /* ORC_INNER_*                                       */
  int inner_fixed;     /* > 0: exactly this many inner iterations           */
  double eps_in;       /* gap mode: stop when FW gap <= eps_in              */
  int inner_check_every;
  int max_inner;
  int outer_fixed;     /* > 0: exactly this many outer iterations           */
  double eps_out;      /* certificate mode tolerance                        */
  int outer_check_every;
  int max_outer;
  int want_last, want_avg;
  int inner_cert_step; /* 1: stop on the step certificate (sigma > 0 only)   */
  int stop_fstar;      /* 1: stop on |F(u) - f_star| <= eps_out instead of   */
  double f_star;       /*    F(u) - d_lb (Sec. 6: the paper's experiments)   */
} orc_opts;

typedef struct {
  int status;          /* 0 converged / fixed run done, 1 not converged     */
  int outer_iters;
  long long inner_iters;
  int converged_last, converged_avg;
  double f_last, infeas_last, f_avg, infeas_avg, d_lb;
} orc_result;

/* ---------------------------------------------------------------- basics */

static double dot(int n, const double *a, const double *b) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

static double clampd(double v, double lo, double hi) {
  return v < lo ? lo : (v > hi ? hi : v);
}

/* y = M v for an m x n row-major matrix M. */
static void matvec(int m, int n, const double *M, const double *v, double *y) {
  for (int r = 0; r < m; ++r) y[r] = dot(n, M + (size_t)r * n, v);
}

/* y = M' v for an m x n row-major matrix M (y has n entries). */
static void matvec_t(int m, int n, const double *M, const double *v, double *y) {
  for (int c = 0; c < n; ++c) y[c] = 0.0;
  for (int r = 0; r < m; ++r)
    for (int c = 0; c < n; ++c) y[c] += M[(size_t)r * n + c] * v[r];
}

/* Projection onto K: R^p_- -> min(z, 0); {0} -> 0  (notation [.]_X, Sec. 1). */
static double proj_K(int cone, double z) {
  if (cone == ORC_CONE_EQ) return 0.0;
  return z < 0.0 ? z : 0.0;
}

/* ------------------------------------------------- problem-level functions */

/* F(u) = 1/2 u'Qu + q'u   (eq. original_primal). */
double orc_F(const orc_qp *qp, const double *u) {
  int n = qp->n;
  double *Qu = malloc(sizeof(double) * n);
  matvec(n, n, qp->Q, u, Qu);
  double f = 0.5 * dot(n, u, Qu) + dot(n, qp->q, u);
  free(Qu);
  return f;
}

/* dist_K(Gu + g) = || Gu + g - [Gu + g]_K ||_2   (notation, Sec. 1). */
double orc_infeas(const orc_qp *qp, const double *u) {
  int p = qp->p;
  if (p == 0) return 0.0;
  double *r = malloc(sizeof(double) * p);
  matvec(p, qp->n, qp->G, u, r);
  double s = 0.0;
  for (int j = 0; j < p; ++j) {
    double z = r[j] + qp->g[j];
    double d = z - proj_K(qp->cone, z);
    s += d * d;
  }
  free(r);
  return sqrt(s);
}

/* Augmented Lagrangian L_rho(u, lambda)   (eq. auglag1). */
double orc_lagrangian(const orc_qp *qp, double rho, const double *u, const double *lam) {
  int p = qp->p;
  double f = orc_F(qp, u);
  if (p == 0) return f;
  double *r = malloc(sizeof(double) * p);
  matvec(p, qp->n, qp->G, u, r);
  double val;
  if (rho > 0.0) {
    /* F(u) + rho/2 dist_K(Gu + g + lambda/rho)^2 - ||lambda||^2 / (2 rho) */
    double d2 = 0.0, l2 = 0.0;
    for (int j = 0; j < p; ++j) {
      double z = r[j] + qp->g[j] + lam[j] / rho;
      double d = z - proj_K(qp->cone, z);
      d2 += d * d;
      l2 += lam[j] * lam[j];
    }
    val = f + 0.5 * rho * d2 - l2 / (2.0 * rho);
  } else {
    /* F(u) + <lambda, Gu + g> */
    double s = 0.0;
    for (int j = 0; j < p; ++j) s += lam[j] * (r[j] + qp->g[j]);
    val = f + s;
  }
  free(r);
  return val;
}

/* s(u, lambda): argmin over s in K of the coupling term   (Sec. 2). */
static void s_of(const orc_qp *qp, double rho, const double *Gu, const double *lam, double *s) {
  for (int j = 0; j < qp->p; ++j) {
    if (rho > 0.0)
      s[j] = proj_K(qp->cone, Gu[j] + qp->g[j] + lam[j] / rho);
    else
      s[j] = 0.0;
  }
}

/* Inexact dual gradient  G u + g - s(u, lambda)   (eq. Ld, eq. inexact_framework). */
void orc_dual_grad(const orc_qp *qp, double rho, const double *u, const double *lam, double *out) {
  int p = qp->p;
  double *Gu = malloc(sizeof(double) * (p ? p : 1));
  double *s = malloc(sizeof(double) * (p ? p : 1));
  matvec(p, qp->n, qp->G, u, Gu);
  s_of(qp, rho, Gu, lam, s);
  for (int j = 0; j < p; ++j) out[j] = Gu[j] + qp->g[j] - s[j];
  free(Gu);
  free(s);
}

/* grad_u L_rho(u, lambda)   (differentiating eq. auglag1):
 *   rho > 0 : Qu + q + G' * rho * (z - [z]_K),  z = Gu + g + lambda/rho
 *   rho = 0 : Qu + q + G' lambda                                          */
void orc_grad_lagr(const orc_qp *qp, double rho, const double *u, const double *lam, double *out) {
  int n = qp->n, p = qp->p;
  matvec(n, n, qp->Q, u, out);
  for (int i = 0; i < n; ++i) out[i] += qp->q[i];
  if (p == 0) return;
  double *Gu = malloc(sizeof(double) * p);
  double *w = malloc(sizeof(double) * p);
  double *Gtw = malloc(sizeof(double) * n);
  matvec(p, n, qp->G, u, Gu);
  for (int j = 0; j < p; ++j) {
    if (rho > 0.0) {
      double z = Gu[j] + qp->g[j] + lam[j] / rho;
      w[j] = rho * (z - proj_K(qp->cone, z));
    } else {
      w[j] = lam[j];
    }
  }
  matvec_t(p, n, qp->G, w, Gtw);
  for (int i = 0; i < n; ++i) out[i] += Gtw[i];
  free(Gu);
  free(w);
  free(Gtw);
}

/* Frank-Wolfe gap of phi = L_rho(., lambda) over the box at x:
 *   max_{v in U} <grad phi(x), x - v>  >=  phi(x) - min_U phi.
 * Reading of the inner criterion eq. duquad_in: this certificate bounds
 * L_rho(x, mu) - d_rho(mu) from above, so gap <= eps_in implies it. */
double orc_fw_gap(const orc_qp *qp, double rho, const double *x, const double *lam) {
  int n = qp->n;
  double *gr = malloc(sizeof(double) * n);
  orc_grad_lagr(qp, rho, x, lam, gr);
  double s = 0.0;
  for (int i = 0; i < n; ++i) {
    double a = gr[i] * qp->lb[i], b = gr[i] * qp->ub[i];
    s += gr[i] * x[i] - (a < b ? a : b);
  }
  free(gr);
  return s;
}

/* Certificate of the inner criterion eq. duquad_in: a computable upper bound
 * on L_rho(x, mu) - d_rho(mu) = phi(x) - phi*.
 *   sigma > 0: with x+ = [x - grad phi(x)/L]_U and g = L (x - x+),
 *       phi(x) - phi* <= <grad phi(x), x - x+> + ||g||^2 (1/(2 sigma) - 1/(2 L))
 *     (convexity bounds phi(x) - phi(x+); the proximal-gradient inequality for
 *     a sigma-strongly convex, L-smooth phi bounds phi(x+) - phi*).  It is a
 *     sum of squares-like terms, robust to rounding of the gradient.
 *   sigma = 0: the Frank-Wolfe gap above.
 * Reading: the paper states the criterion through the unknown d_rho(mu); any
 * computable upper bound on it enforces eq. duquad_in. */
double orc_inner_cert(const orc_qp *qp, double rho, const double *x, const double *lam,
                      double LL, double sigma) {
  if (!(sigma > 0.0)) return orc_fw_gap(qp, rho, x, lam);
  int n = qp->n;
  double *gr = malloc(sizeof(double) * n);
  orc_grad_lagr(qp, rho, x, lam, gr);
  double kappa = 1.0 / (2.0 * sigma) - 1.0 / (2.0 * LL);
  double lin = 0.0, sq = 0.0;
  for (int i = 0; i < n; ++i) {
    double xp = clampd(x[i] - gr[i] / LL, qp->lb[i], qp->ub[i]);
    double d = x[i] - xp;
    lin += gr[i] * d;
    sq += (LL * d) * (LL * d);
  }
  free(gr);
  return lin + sq * kappa;
}

/* Step certificate: a bound for the iterate x+ = [y - grad phi(y)/L]_U that
 * a gradient step from ANY point y (inside the box or not) produces,
 *     phi(x+) - phi* <= ||g||^2 (1/(2 sigma) - 1/(2 L)),  g = L (y - x+),
 * the proximal-gradient inequality for a sigma-strongly convex, L-smooth phi
 * (the second half of the bound above, taken at the step point instead of at
 * the iterate).  It needs only y and x+, which the inner step forms anyway,
 * so an implementation can check it every iteration without another
 * gradient.  Reading: any computable upper bound on L_rho(x, mu) - d_rho(mu)
 * enforces eq. duquad_in; this one is defined for sigma > 0 only.
 * xplus (optional) receives x+. */
double orc_step_cert(const orc_qp *qp, double rho, const double *y, const double *lam,
                     double LL, double sigma, double *xplus) {
  int n = qp->n;
  double *gr = malloc(sizeof(double) * n);
  orc_grad_lagr(qp, rho, y, lam, gr);
  double sq = 0.0;
  for (int i = 0; i < n; ++i) {
    double xp = clampd(y[i] - gr[i] / LL, qp->lb[i], qp->ub[i]);
    if (xplus) xplus[i] = xp;
    double g = LL * (y[i] - xp);
    sq += g * g;
  }
  free(gr);
  return sq * (1.0 / (2.0 * sigma) - 1.0 / (2.0 * LL));
}

/* ---------------------------------------------------- Algorithm FOM (inner) */

/* Algorithm FOM(phi, X) of Sec. 2.1 with phi = L_rho(., mu), X = U:
 *   given x^0 = y^1 in X, for k >= 1:
 *     x^k     = [ y^k - grad phi(y^k) / L_phi ]_X
 *     y^{k+1} = x^k + beta_k (x^k - x^{k-1})
 *   GM: beta_k = 0; FGM: beta_k = (theta_k - 1)/theta_{k+1},
 *   theta_{k+1} = (1 + sqrt(1 + 4 theta_k^2))/2, theta_1 = 1;
 *   FGM_sigma: beta_k = (sqrt(L) - sqrt(sigma)) / (sqrt(L) + sqrt(sigma)).
 * x holds x^0 on entry and the returned iterate on exit.
 * Stops after exactly inner_fixed iterations, or (certificate mode) at the
 * first k that is a multiple of inner_check_every with cert(x^k) <= eps_in, or
 * at max_inner.  cert is orc_inner_cert at x^k, or (cert_step, sigma > 0)
 * orc_step_cert of the step y^k -> x^k.  Returns the number of iterations
 * performed.
 * phi_trace (optional, length >= cap) receives phi(x^k) for k = 1.. */
int orc_fom(const orc_qp *qp, double rho, const double *mu, double LL, double sigma,
            int variant, int inner_fixed, double eps_in, int check_every, int max_inner,
            int cert_step, double *x, double *phi_trace, int cap) {
  int n = qp->n;
  double *xp = malloc(sizeof(double) * n);  /* x^{k-1} */
  double *y = malloc(sizeof(double) * n);   /* y^k     */
  double *xn = malloc(sizeof(double) * n);  /* x^k     */
  double *gr = malloc(sizeof(double) * n);
  memcpy(xp, x, sizeof(double) * n);
  memcpy(y, x, sizeof(double) * n);
  if (variant == ORC_INNER_AUTO) variant = sigma > 0.0 ? ORC_INNER_FGMSIGMA : ORC_INNER_FGM;
  double beta_sigma = (sqrt(LL) - sqrt(sigma)) / (sqrt(LL) + sqrt(sigma));
  double theta = 1.0;
  if (check_every < 1) check_every = 1;
  int k = 0;
  for (;;) {
    ++k;
    orc_grad_lagr(qp, rho, y, mu, gr);
    for (int i = 0; i < n; ++i) xn[i] = clampd(y[i] - gr[i] / LL, qp->lb[i], qp->ub[i]);
    /* step certificate of y^k -> x^k, before y moves on */
    double cstep = (cert_step && sigma > 0.0 && inner_fixed <= 0 && k % check_every == 0)
                       ? orc_step_cert(qp, rho, y, mu, LL, sigma, NULL)
                       : 0.0;
    double beta;
    if (variant == ORC_INNER_GM) {
      beta = 0.0;
    } else if (variant == ORC_INNER_FGM) {
      double theta_next = 0.5 * (1.0 + sqrt(1.0 + 4.0 * theta * theta));
      beta = (theta - 1.0) / theta_next;
      theta = theta_next;
    } else {
      beta = beta_sigma;
    }
    for (int i = 0; i < n; ++i) y[i] = xn[i] + beta * (xn[i] - xp[i]);
    memcpy(xp, xn, sizeof(double) * n);
    if (phi_trace && k <= cap) phi_trace[k - 1] = orc_lagrangian(qp, rho, xn, mu);
    if (inner_fixed > 0) {
      if (k >= inner_fixed) break;
    } else {
      if (k % check_every == 0) {
        double cert = (cert_step && sigma > 0.0) ? cstep : orc_inner_cert(qp, rho, xn, mu, LL, sigma);
        if (cert <= eps_in) break;
      }
      if (k >= max_inner) break;
    }
  }
  memcpy(x, xn, sizeof(double) * n);
  free(xp);
  free(y);
  free(xn);
  free(gr);
  return k;
}

/* ------------------------------------------------ Algorithm DFOM (outer) */

static int is_fast(int alg) { return alg == ORC_DFGM || alg == ORC_ADFGM; }

/* [z]_{K_d}: K_d = R^p_+ for K = R^p_- (reading: also when Q is singular,
 * unless kd_literal asks for the paper's literal R^p there), R^p for K = {0}
 * (Sec. 2, definition of K_d). */
static double proj_Kd(const orc_qp *qp, const orc_opts *o, double z) {
  if (qp->cone == ORC_CONE_EQ) return z;
  if (o->kd_literal && !(o->sigma > 0.0)) return z;
  return z > 0.0 ? z : 0.0;
}

static int lower_bound_valid(const orc_qp *qp, const orc_opts *o, const double *mu) {
  /* d_rho(mu) <= F* holds for every mu when rho > 0 or K = {0}; for rho = 0
   * and K = R^p_- it needs mu >= 0 (weak duality). */
  if (o->rho > 0.0 || qp->cone == ORC_CONE_EQ) return 1;
  for (int j = 0; j < qp->p; ++j)
    if (mu[j] < 0.0) return 0;
  return 1;
}

/* Algorithm DFOM(d_rho, K_d) of Sec. 3 with primal outputs of Sec. 4:
 *   given lambda^0 = mu^1 in K_d, theta_1 = 1, for k >= 1:
 *     ubar^k    = FOM(L_rho(., mu^k), U), warm-started from ubar^{k-1}
 *     lambda^k  = [ mu^k + (1/(2 L_d)) (G ubar^k + g - s(ubar^k, mu^k)) ]_{K_d}
 *     mu^{k+1}  = lambda^k + beta_k (lambda^k - lambda^{k-1})
 *   DGM: beta_k = 0; DFGM: theta-rule as in FOM.
 *   average output  uhat^k = sum_{j=1}^k theta_j ubar^j / S_k (eq. average_primal)
 *   last output     ubar(lambda^k): equals ubar^k for DGM/ADGM (reading of
 *                   eq. last_primal); one extra warm-started inner solve at
 *                   mu = lambda^k for DFGM/ADFGM.
 * Stopping: fixed outer count, or the certificate read from Sec. 3.1 and the
 * epsilon-primal definition: dist_K(Gu + g) <= eps_out and F(u) - d_lb <= eps_out,
 * d_lb = max over checked outers of L_rho(ubar, mu) - cert (a lower bound of F*);
 * or, as in the paper's experiments (Sec. 6) with F* known, |F(u) - F*| <= eps_out
 * in place of F(u) - d_lb <= eps_out (stop_fstar).
 * trace (optional) receives ORC_TRACE_COLS values per outer iteration.      */
int orc_dfom(const orc_qp *qp, const orc_opts *o, const double *lambda0, const double *x0,
             double *x_last, double *x_avg, double *lambda_out, orc_result *res,
             double *trace, int trace_cap) {
  int n = qp->n, p = qp->p;
  int pp = p ? p : 1;
  double rho = o->rho;
  double alpha = 1.0 / (2.0 * o->Ld);
  double *u = malloc(sizeof(double) * n);      /* ubar^k (warm start chain)  */
  double *ul = malloc(sizeof(double) * n);     /* ubar(lambda^k) (DFGM last) */
  double *usum = calloc(n, sizeof(double));    /* sum theta_j ubar^j         */
  double *uavg = malloc(sizeof(double) * n);
  double *lam = malloc(sizeof(double) * pp);   /* lambda^k                   */
  double *lamp = malloc(sizeof(double) * pp);  /* lambda^{k-1}               */
  double *mu = malloc(sizeof(double) * pp);    /* mu^k                       */
  double *dg = malloc(sizeof(double) * pp);
  memset(res, 0, sizeof(*res));
  res->d_lb = -INFINITY;
  res->f_last = res->f_avg = res->infeas_last = res->infeas_avg = NAN;

  for (int i = 0; i < n; ++i)
    u[i] = x0 ? x0[i] : clampd(0.0, qp->lb[i], qp->ub[i]);
  for (int j = 0; j < p; ++j) {
    lamp[j] = lambda0 ? lambda0[j] : 0.0;
    lam[j] = lamp[j];
    mu[j] = lamp[j];
  }
  double theta = 1.0, S = 0.0;
  long long inner_total = 0;
  int fast = is_fast(o->alg);
  int check_every = o->outer_check_every > 0 ? o->outer_check_every : 1;
  int kmax = o->outer_fixed > 0 ? o->outer_fixed : o->max_outer;
  int k = 0, converged = 0;

  while (k < kmax && !converged) {
    ++k;
    /* step 1: inner solve at mu^k, warm start from ubar^{k-1} */
    int it = orc_fom(qp, rho, mu, o->LL, o->sigma, o->inner_variant, o->inner_fixed, o->eps_in,
                     o->inner_check_every, o->max_inner, o->inner_cert_step, u, NULL, 0);
    inner_total += it;
    /* step 2: inexact dual gradient and projected dual step */
    orc_dual_grad(qp, rho, u, mu, dg);
    for (int j = 0; j < p; ++j) lam[j] = proj_Kd(qp, o, mu[j] + alpha * dg[j]);
    /* averaging weight theta_k, then the momentum step 3 */
    S += theta;
    for (int i = 0; i < n; ++i) usum[i] += theta * u[i];
    double beta = 0.0, theta_k = theta;
    if (fast) {
      double theta_next = 0.5 * (1.0 + sqrt(1.0 + 4.0 * theta * theta));
      beta = (theta - 1.0) / theta_next;
      theta = theta_next;
    }
    if (trace && k <= trace_cap) {
      double *t = trace + (size_t)(k - 1) * ORC_TRACE_COLS;
      double mnl = INFINITY, nl = 0.0;
      for (int j = 0; j < p; ++j) {
        if (lam[j] < mnl) mnl = lam[j];
        nl += lam[j] * lam[j];
      }
      t[0] = k;
      t[1] = theta_k;
      t[2] = S;
      t[3] = beta;
      t[4] = it;
      t[5] = orc_lagrangian(qp, rho, u, mu); /* dbar_rho(mu^k) */
      t[6] = dot(p, dg, mu);                 /* <grad dbar, mu^k> */
      t[7] = orc_F(qp, u);
      t[8] = dot(p, dg, dg);
      t[9] = p ? mnl : 0.0;
      t[10] = sqrt(nl);
      t[11] = orc_infeas(qp, u);
    }
    int final_iter = (k == kmax);
    int check = final_iter || (o->outer_fixed <= 0 && k % check_every == 0);
    if (check) {
      /* lower bound from this outer's inner solution */
      if (lower_bound_valid(qp, o, mu)) {
        double lb = orc_lagrangian(qp, rho, u, mu) - orc_inner_cert(qp, rho, u, mu, o->LL, o->sigma);
        if (lb > res->d_lb) res->d_lb = lb;
      }
      if (o->want_last) {
        memcpy(ul, u, sizeof(double) * n);
        if (fast) {
          int it2 = orc_fom(qp, rho, lam, o->LL, o->sigma, o->inner_variant, o->inner_fixed,
                            o->eps_in, o->inner_check_every, o->max_inner, o->inner_cert_step, ul,
                            NULL, 0);
          inner_total += it2;
          if (lower_bound_valid(qp, o, lam)) {
            double lb = orc_lagrangian(qp, rho, ul, lam) - orc_inner_cert(qp, rho, ul, lam, o->LL, o->sigma);
            if (lb > res->d_lb) res->d_lb = lb;
          }
        }
        res->f_last = orc_F(qp, ul);
        res->infeas_last = orc_infeas(qp, ul);
      }
      if (o->want_avg) {
        for (int i = 0; i < n; ++i) uavg[i] = usum[i] / S;
        res->f_avg = orc_F(qp, uavg);
        res->infeas_avg = orc_infeas(qp, uavg);
      }
      if (o->outer_fixed <= 0) {
        double gap_last = res->f_last - res->d_lb, gap_avg = res->f_avg - res->d_lb;
        if (o->stop_fstar) {
          gap_last = fabs(res->f_last - o->f_star);
          gap_avg = fabs(res->f_avg - o->f_star);
        }
        res->converged_last = o->want_last && res->infeas_last <= o->eps_out && gap_last <= o->eps_out;
        res->converged_avg = o->want_avg && res->infeas_avg <= o->eps_out && gap_avg <= o->eps_out;
        converged = res->converged_last || res->converged_avg;
      }
    }
    for (int j = 0; j < p; ++j) {
      double m = lam[j] + beta * (lam[j] - lamp[j]);
      lamp[j] = lam[j];
      mu[j] = m;
    }
  }
  if (!o->want_last) memcpy(ul, u, sizeof(double) * n);
  res->outer_iters = k;
  res->inner_iters = inner_total;
  res->status = (o->outer_fixed > 0 || converged) ? 0 : 1;
  if (x_last) memcpy(x_last, ul, sizeof(double) * n);
  if (x_avg) {
    for (int i = 0; i < n; ++i) uavg[i] = usum[i] / S;
    memcpy(x_avg, uavg, sizeof(double) * n);
  }
  if (lambda_out) memcpy(lambda_out, lam, sizeof(double) * p);
  free(u);
  free(ul);
  free(usum);
  free(uavg);
  free(lam);
  free(lamp);
  free(mu);
  free(dg);
  return res->status;
}

/* ------------------------------------------------------------- constants */

/* Power iteration for lambda_max of the symmetric PSD operator v -> A v,
 * A = Q (which = 0) or A = G'G (which = 1, giving ||G||^2).  The constants
 * L_L = lambda_max(Q) + rho ||G||^2 and L_d = ||G||^2/(lambda_min(Q) + rho ||G||^2)
 * are the ones of eq. Ld and Step 1 of Sec. 3.  Returns the Rayleigh quotient
 * after iters steps from the all-ones start vector. */
double orc_power_lmax(const orc_qp *qp, int which, int iters) {
  int n = qp->n, p = qp->p;
  double *v = malloc(sizeof(double) * n);
  double *w = malloc(sizeof(double) * n);
  double *t = malloc(sizeof(double) * (p ? p : 1));
  for (int i = 0; i < n; ++i) v[i] = 1.0 / sqrt((double)n);
  double ray = 0.0;
  for (int it = 0; it < iters; ++it) {
    if (which == 0) {
      matvec(n, n, qp->Q, v, w);
    } else {
      matvec(p, n, qp->G, v, t);
      matvec_t(p, n, qp->G, t, w);
    }
    ray = dot(n, v, w);
    double nw = sqrt(dot(n, w, w));
    if (nw == 0.0) break;
    for (int i = 0; i < n; ++i) v[i] = w[i] / nw;
  }
  free(v);
  free(w);
  free(t);
  return ray;
}
