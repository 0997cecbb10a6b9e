// sparse.cu -- problem handles for sparse (CSR) Q and G.
//
// Sec. 5 notes that the method needs only matrix-vector products, so for
// sparse Q and G (e.g. network utility maximisation) each iteration costs
// O(nnz).  This file validates a CSR problem on the host, builds the CSR of
// G' by a stable counting sort (so every product sums its row in a fixed
// order), computes the guaranteed spectral bounds when asked, and uploads the
// arrays; the grid engine runs the solve with CSR products (csr.cuh).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "dq_host.h"

namespace dq {

namespace {

struct HostCsr {
  int rows = 0, cols = 0;
  std::vector<int> rp, ci;
  std::vector<double> val;
};

// Copy one CSR matrix (host or device arrays) into host vectors.
dq_status fetch_csr(int rows, int cols, int nnz, const int* rp, const int* ci, const void* val, int memory,
                    size_t esz, HostCsr* out, const char* name) {
  if (nnz < 0 || (rows > 0 && !rp) || (nnz > 0 && (!ci || !val))) {
    set_error("%s: NULL CSR array or negative nnz", name);
    return DQ_ERR_INVALID;
  }
  out->rows = rows;
  out->cols = cols;
  out->rp.resize((size_t)rows + 1);
  out->ci.resize((size_t)nnz);
  out->val.resize((size_t)nnz);
  if (memory == DQ_HOST) {
    memcpy(out->rp.data(), rp, ((size_t)rows + 1) * 4);
    if (nnz) {
      memcpy(out->ci.data(), ci, (size_t)nnz * 4);
      memcpy(out->val.data(), val, (size_t)nnz * 8);
    }
  } else {
    DQ_CK(cudaMemcpy(out->rp.data(), rp, ((size_t)rows + 1) * 4, cudaMemcpyDeviceToHost));
    if (nnz) {
      DQ_CK(cudaMemcpy(out->ci.data(), ci, (size_t)nnz * 4, cudaMemcpyDeviceToHost));
      if (esz == 8) {
        DQ_CK(cudaMemcpy(out->val.data(), val, (size_t)nnz * 8, cudaMemcpyDeviceToHost));
      } else {
        std::vector<float> f((size_t)nnz);
        DQ_CK(cudaMemcpy(f.data(), val, (size_t)nnz * 4, cudaMemcpyDeviceToHost));
        for (size_t e = 0; e < f.size(); ++e) out->val[e] = f[e];
      }
    }
  }
  // structure and values
  if (out->rp[0] != 0 || out->rp[rows] != nnz) {
    set_error("%s: rowptr[0] must be 0 and rowptr[rows] = nnz", name);
    return DQ_ERR_INVALID;
  }
  for (int r = 0; r < rows; ++r) {
    const int e0 = out->rp[r], e1 = out->rp[r + 1];
    if (e1 < e0) {
      set_error("%s: row offsets decrease at row %d", name, r);
      return DQ_ERR_INVALID;
    }
    for (int e = e0; e < e1; ++e) {
      const int c = out->ci[e];
      if (c < 0 || c >= cols || (e > e0 && c <= out->ci[e - 1])) {
        set_error("%s: row %d: column indices out of range or not strictly increasing", name, r);
        return DQ_ERR_INVALID;
      }
      if (!std::isfinite(out->val[e])) {
        set_error("non-finite value in %s", name);
        return DQ_ERR_INVALID;
      }
    }
  }
  return DQ_OK;
}

// CSR of the transpose, rows in increasing order within each column (stable).
HostCsr transpose(const HostCsr& A) {
  HostCsr T;
  T.rows = A.cols;
  T.cols = A.rows;
  T.rp.assign((size_t)A.cols + 1, 0);
  for (int c : A.ci) ++T.rp[(size_t)c + 1];
  for (int c = 0; c < A.cols; ++c) T.rp[c + 1] += T.rp[c];
  T.ci.resize(A.ci.size());
  T.val.resize(A.val.size());
  std::vector<int> pos(T.rp.begin(), T.rp.end() - 1);
  for (int r = 0; r < A.rows; ++r)
    for (int e = A.rp[r]; e < A.rp[r + 1]; ++e) {
      const int d = pos[A.ci[e]]++;
      T.ci[d] = r;
      T.val[d] = A.val[e];
    }
  return T;
}

dq_status fetch_vec(const void* src, size_t m, int memory, size_t esz, std::vector<double>* out, const char* name) {
  out->resize(m);
  if (m == 0) return DQ_OK;
  if (!src) {
    set_error("NULL vector %s", name);
    return DQ_ERR_INVALID;
  }
  if (memory == DQ_HOST) {
    memcpy(out->data(), src, m * 8);
  } else if (esz == 8) {
    DQ_CK(cudaMemcpy(out->data(), src, m * 8, cudaMemcpyDeviceToHost));
  } else {
    std::vector<float> f(m);
    DQ_CK(cudaMemcpy(f.data(), src, m * 4, cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < m; ++i) (*out)[i] = f[i];
  }
  for (double v : *out)
    if (!std::isfinite(v)) {
      set_error("non-finite value in %s", name);
      return DQ_ERR_INVALID;
    }
  return DQ_OK;
}

// Device copy of host data in the element type (esz 8: double, 4: float).
dq_status put(void** dst, const void* src, size_t bytes) {
  if (bytes == 0) return DQ_OK;
  if (cudaMalloc(dst, bytes) != cudaSuccess) {
    cudaGetLastError();
    *dst = nullptr;
    set_error("device allocation of %zu bytes failed", bytes);
    return DQ_ERR_NOMEM;
  }
  DQ_CK(cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice));
  return DQ_OK;
}

dq_status put_vals(void** dst, const std::vector<double>& v, size_t esz) {
  if (esz == 8) return put(dst, v.data(), v.size() * 8);
  std::vector<float> f(v.begin(), v.end());
  return put(dst, f.data(), f.size() * 4);
}

}  // namespace

}  // namespace dq

using namespace dq;

extern "C" dq_status dq_problem_create_sparse(dq_context* ctx, const dq_sparse_desc* d, dq_problem** out) {
  if (!ctx || !d || !out) {
    set_error("NULL argument");
    return DQ_ERR_INVALID;
  }
  *out = nullptr;
  if (d->n < 1 || d->p < 0) {
    set_error("need n >= 1, p >= 0 (got %d, %d)", d->n, d->p);
    return DQ_ERR_INVALID;
  }
  if ((d->cone != DQ_CONE_INEQ && d->cone != DQ_CONE_EQ) || (d->prec != DQ_FP64 && d->prec != DQ_FP32) ||
      (d->memory != DQ_HOST && d->memory != DQ_DEVICE) ||
      (d->lipschitz != DQ_LIP_LANCZOS && d->lipschitz != DQ_LIP_BOUND)) {
    set_error("sparse problem: bad cone, precision (DQ_FP64 or DQ_FP32), memory or lipschitz mode");
    return DQ_ERR_INVALID;
  }
  if (!std::isnan(d->lmin_Q) && d->lmin_Q < 0) {
    set_error("lmin_Q must be a lower bound >= 0");
    return DQ_ERR_INVALID;
  }
  DQ_CK(cudaSetDevice(ctx->device));
  const size_t esz = d->prec == DQ_FP64 ? 8 : 4;
  const int n = d->n, p = d->p;
  HostCsr Q, G;
  dq_status s;
  if ((s = fetch_csr(n, n, d->nnz_Q, d->Q_rowptr, d->Q_col, d->Q_val, d->memory, esz, &Q, "Q")) != DQ_OK) return s;
  if (p > 0) {
    if ((s = fetch_csr(p, n, d->nnz_G, d->G_rowptr, d->G_col, d->G_val, d->memory, esz, &G, "G")) != DQ_OK)
      return s;
  } else {
    G.rows = 0;
    G.cols = n;
    G.rp.assign(1, 0);
  }
  std::vector<double> q, g, lb, ub;
  if ((s = fetch_vec(d->q, n, d->memory, esz, &q, "q")) != DQ_OK ||
      (s = fetch_vec(d->g, p, d->memory, esz, &g, "g")) != DQ_OK ||
      (s = fetch_vec(d->lb, n, d->memory, esz, &lb, "lb")) != DQ_OK ||
      (s = fetch_vec(d->ub, n, d->memory, esz, &ub, "ub")) != DQ_OK)
    return s;
  for (int i = 0; i < n; ++i)
    if (!(lb[i] <= ub[i])) {
      set_error("lb > ub for some coordinate");
      return DQ_ERR_INVALID;
    }
  // symmetry: Q' has the same structure and (within the tolerance) the same values
  const HostCsr Qt = transpose(Q);
  std::vector<double> diag(n, 0.0);
  for (int r = 0; r < n; ++r)
    for (int e = Q.rp[r]; e < Q.rp[r + 1]; ++e)
      if (Q.ci[e] == r) diag[r] = Q.val[e];
  const double tol = d->prec == DQ_FP64 ? 1e-10 : 1e-6;
  if (Qt.rp != Q.rp || Qt.ci != Q.ci) {
    set_error("Q is not symmetric (its sparsity pattern differs from its transpose's)");
    return DQ_ERR_INVALID;
  }
  for (int r = 0; r < n; ++r)
    for (int e = Q.rp[r]; e < Q.rp[r + 1]; ++e) {
      const int c = Q.ci[e];
      if (!(fabs(Q.val[e] - Qt.val[e]) <= tol * sqrt(fabs(diag[r] * diag[c])))) {
        set_error("Q is not symmetric: |Q[%d][%d] - Q[%d][%d]| exceeds the tolerance", r, c, c, r);
        return DQ_ERR_INVALID;
      }
    }
  const HostCsr Gt = transpose(G);
  dq_problem* P = new dq_problem();
  P->ctx = ctx;
  ++ctx->live_problems;
  P->n = n;
  P->p = p;
  P->batch = 1;
  P->cone = d->cone;
  P->prec = d->prec;
  P->esz = esz;
  P->sparse = true;
  P->own_Q = P->own_G = true;
  P->nnzQ = (long long)Q.ci.size();
  P->nnzG = (long long)G.ci.size();
  P->lmin_Q = d->lmin_Q;
  P->lmax_Q = P->lmax_given = d->lmax_Q;
  P->normG2 = P->normG2_given = d->normG2;
  P->lip_bound = d->lipschitz == DQ_LIP_BOUND;
  if (P->lip_bound) {  // the guaranteed bounds of dq_lipschitz from the host CSR (FP64)
    double gersh = 0.0, fro = 0.0;
    for (int r = 0; r < n; ++r) {
      double s1 = 0.0;
      for (int e = Q.rp[r]; e < Q.rp[r + 1]; ++e) {
        s1 += fabs(Q.val[e]);
        fro += Q.val[e] * Q.val[e];
      }
      gersh = std::max(gersh, s1);
    }
    if (std::isnan(P->lmax_Q)) P->lmax_Q = P->lmax_given = std::min(gersh, sqrt(fro));
    double n1 = 0.0, ninf = 0.0, gf = 0.0;
    for (int r = 0; r < p; ++r) {
      double s1 = 0.0;
      for (int e = G.rp[r]; e < G.rp[r + 1]; ++e) {
        s1 += fabs(G.val[e]);
        gf += G.val[e] * G.val[e];
      }
      ninf = std::max(ninf, s1);
    }
    for (int c = 0; c < n; ++c) {
      double s1 = 0.0;
      for (int e = Gt.rp[c]; e < Gt.rp[c + 1]; ++e) s1 += fabs(Gt.val[e]);
      n1 = std::max(n1, s1);
    }
    if (std::isnan(P->normG2)) P->normG2 = P->normG2_given = std::min(n1 * ninf, gf);
  }
  auto fail = [&](dq_status st) {
    dq_problem_destroy(P);
    return st;
  };
  const size_t pn = std::max(p, 1);
  if ((s = put_vals(&P->Q, Q.val, esz)) != DQ_OK || (s = put((void**)&P->q_rp, Q.rp.data(), Q.rp.size() * 4)) != DQ_OK ||
      (s = put((void**)&P->q_ci, Q.ci.data(), Q.ci.size() * 4)) != DQ_OK)
    return fail(s);
  if (p > 0) {
    if ((s = put_vals(&P->G, G.val, esz)) != DQ_OK ||
        (s = put((void**)&P->g_rp, G.rp.data(), G.rp.size() * 4)) != DQ_OK ||
        (s = put((void**)&P->g_ci, G.ci.data(), G.ci.size() * 4)) != DQ_OK ||
        (s = put_vals(&P->GT, Gt.val, esz)) != DQ_OK ||
        (s = put((void**)&P->gt_rp, Gt.rp.data(), Gt.rp.size() * 4)) != DQ_OK ||
        (s = put((void**)&P->gt_ci, Gt.ci.data(), Gt.ci.size() * 4)) != DQ_OK ||
        (s = put_vals(&P->g, g, esz)) != DQ_OK)
      return fail(s);
  }
  if ((s = put_vals(&P->q, q, esz)) != DQ_OK || (s = put_vals(&P->lb, lb, esz)) != DQ_OK ||
      (s = put_vals(&P->ub, ub, esz)) != DQ_OK)
    return fail(s);
  std::vector<double> zn(n, 0.0), zp(pn, 0.0);
  if ((s = put_vals(&P->x_state, zn, esz)) != DQ_OK || (s = put_vals(&P->lam_state, zp, esz)) != DQ_OK)
    return fail(s);
  *out = P;
  return DQ_OK;
}
