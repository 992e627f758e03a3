// Host set-up, part 2: non-nested transfer, sparse products, dense SPD inverses and
// the largest eigenvalue of the Jacobi-scaled operator.
//
// Transfer (Sec. 2, Eq. 2): [P_l]_ij = phi_j^{(l+1)}(x_i). Each free fine DoF point is
// located in the coarse mesh through a uniform bucket grid: the lowest-numbered coarse
// cell whose barycentric coordinates at the point are all >= -1e-12 is taken, the coarse
// basis is evaluated at the raw barycentric coordinates, and |values| < 1e-14 are dropped.
// Galerkin (Eq. 3): A_{l+1} = R (A P) with R = P^T, row-wise (Gustavson) products.
// Eigenvalue (Sec. 3.2, Sec. 5): Lanczos on D^{-1/2} A D^{-1/2}, optionally restricted to
// the DoFs outside the patches (adjusted lambda_max).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>

#include "internal.hpp"

namespace nnmg {

namespace {

const int kEdges2[3][2] = {{0, 1}, {0, 2}, {1, 2}};
const int kEdges3[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};

// Coarse basis values at barycentric coordinates lam[d+1].
int basis_at(int degree, int d, const double* lam, double* out) {
  if (degree == 1) {
    for (int a = 0; a <= d; ++a) out[a] = lam[a];
    return d + 1;
  }
  for (int a = 0; a <= d; ++a) out[a] = lam[a] * (2.0 * lam[a] - 1.0);
  const int(*le)[2] = d == 2 ? kEdges2 : kEdges3;
  int ne = d == 2 ? 3 : 6;
  for (int e = 0; e < ne; ++e) out[d + 1 + e] = 4.0 * lam[le[e][0]] * lam[le[e][1]];
  return d + 1 + ne;
}

// Barycentric coordinates of point p in cell c.
void barycentric(const MeshH& m, int64_t c, const double* p, double* lam) {
  const int d = m.dim;
  const int32_t* cv = &m.c[c * (d + 1)];
  const double* x0 = &m.x[(int64_t)cv[0] * d];
  double J[3][3], r[3];
  for (int i = 0; i < d; ++i) {
    r[i] = p[i] - x0[i];
    for (int k = 0; k < d; ++k) J[i][k] = m.x[(int64_t)cv[k + 1] * d + i] - x0[i];
  }
  if (d == 2) {
    double det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    lam[1] = (J[1][1] * r[0] - J[0][1] * r[1]) / det;
    lam[2] = (-J[1][0] * r[0] + J[0][0] * r[1]) / det;
    lam[0] = 1.0 - lam[1] - lam[2];
  } else {
    // Cramer's rule
    auto det3 = [](double a[3][3]) {
      return a[0][0] * (a[1][1] * a[2][2] - a[1][2] * a[2][1]) - a[0][1] * (a[1][0] * a[2][2] - a[1][2] * a[2][0]) +
             a[0][2] * (a[1][0] * a[2][1] - a[1][1] * a[2][0]);
    };
    double det = det3(J);
    for (int k = 0; k < 3; ++k) {
      double Jk[3][3];
      std::memcpy(Jk, J, sizeof(J));
      for (int i = 0; i < 3; ++i) Jk[i][k] = r[i];
      lam[k + 1] = det3(Jk) / det;
    }
    lam[0] = 1.0 - lam[1] - lam[2] - lam[3];
  }
}

}  // namespace

Csr prolongation(const DofMapH& fine, const MeshH& cm, const DofMapH& coarse) {
  const int d = cm.dim, d1 = d + 1;
  const double kLocate = -1e-12, kDrop = 1e-14;
  // bucket grid over the coarse bounding box
  double lo[3], hi[3];
  for (int r = 0; r < d; ++r) lo[r] = std::numeric_limits<double>::max(), hi[r] = -lo[r];
  for (int64_t v = 0; v < cm.nv; ++v)
    for (int r = 0; r < d; ++r) lo[r] = std::min(lo[r], cm.x[v * d + r]), hi[r] = std::max(hi[r], cm.x[v * d + r]);
  int64_t nb = std::max<int64_t>(1, (int64_t)std::llround(std::pow((double)cm.nc / 2.0, 1.0 / d)));
  double w[3];
  for (int r = 0; r < d; ++r) w[r] = (hi[r] - lo[r]) / nb + 1e-300;
  auto bidx = [&](double x, int r) {
    int64_t b = (int64_t)std::floor((x - lo[r]) / w[r]);
    return std::min<int64_t>(nb - 1, std::max<int64_t>(0, b));
  };
  int64_t nbt = 1;
  for (int r = 0; r < d; ++r) nbt *= nb;
  std::vector<int64_t> bstart(nbt + 1, 0);
  auto for_cell_buckets = [&](int64_t c, const std::function<void(int64_t)>& f) {
    int64_t b0[3], b1[3];
    for (int r = 0; r < d; ++r) {
      double mn = std::numeric_limits<double>::max(), mx = -mn;
      for (int j = 0; j < d1; ++j) {
        double x = cm.x[(int64_t)cm.c[c * d1 + j] * d + r];
        mn = std::min(mn, x), mx = std::max(mx, x);
      }
      b0[r] = bidx(mn, r), b1[r] = bidx(mx, r);
    }
    if (d == 2) {
      for (int64_t j = b0[1]; j <= b1[1]; ++j)
        for (int64_t i = b0[0]; i <= b1[0]; ++i) f(j * nb + i);
    } else {
      for (int64_t k = b0[2]; k <= b1[2]; ++k)
        for (int64_t j = b0[1]; j <= b1[1]; ++j)
          for (int64_t i = b0[0]; i <= b1[0]; ++i) f((k * nb + j) * nb + i);
    }
  };
  for (int64_t c = 0; c < cm.nc; ++c) for_cell_buckets(c, [&](int64_t b) { bstart[b + 1]++; });
  for (int64_t b = 0; b < nbt; ++b) bstart[b + 1] += bstart[b];
  std::vector<int64_t> bcells(bstart[nbt]), fill(bstart.begin(), bstart.end() - 1);
  for (int64_t c = 0; c < cm.nc; ++c) for_cell_buckets(c, [&](int64_t b) { bcells[fill[b]++] = c; });

  const int nloc = coarse.nloc;
  const int64_t nrows = fine.nfree;
  std::vector<int32_t> cnt(nrows, 0), tc((size_t)nrows * nloc);
  std::vector<double> tv((size_t)nrows * nloc);
  std::vector<uint8_t> failed(nrows, 0);
  parallel_for(nrows, [&](int64_t rlo, int64_t rhi) {
    for (int64_t i = rlo; i < rhi; ++i) {
      const double* p = &fine.points[fine.free_list[i] * d];
      int64_t b = 0;
      if (d == 2) b = bidx(p[1], 1) * nb + bidx(p[0], 0);
      else b = (bidx(p[2], 2) * nb + bidx(p[1], 1)) * nb + bidx(p[0], 0);
      int64_t found = -1;
      double lam[4];
      for (int64_t k = bstart[b]; k < bstart[b + 1]; ++k) {
        int64_t c = bcells[k];
        barycentric(cm, c, p, lam);
        double mn = lam[0];
        for (int j = 1; j < d1; ++j) mn = std::min(mn, lam[j]);
        if (mn >= kLocate) {
          found = c;
          break;
        }
      }
      if (found < 0) {
        failed[i] = 1;
        continue;
      }
      // barycentric coordinates within the location tolerance of zero are exact zeros
      for (int j = 0; j < d1; ++j)
        if (std::fabs(lam[j]) <= -kLocate) lam[j] = 0.0;
      double vals[10];
      basis_at(coarse.degree, d, lam, vals);
      std::pair<int32_t, double> e[10];
      int n = 0;
      for (int a = 0; a < nloc; ++a) {
        int64_t col = coarse.free_index[coarse.cell_dofs[found * nloc + a]];
        if (col < 0 || std::fabs(vals[a]) < kDrop) continue;
        e[n++] = {(int32_t)col, vals[a]};
      }
      std::sort(e, e + n, [](const std::pair<int32_t, double>& a, const std::pair<int32_t, double>& b) {
        return a.first < b.first;
      });
      cnt[i] = n;
      for (int k = 0; k < n; ++k) tc[i * nloc + k] = e[k].first, tv[i * nloc + k] = e[k].second;
    }
  });
  for (int64_t i = 0; i < nrows; ++i)
    if (failed[i]) throw Error(MG_ERR_POINT_LOCATION, "fine DoF " + std::to_string(i) + " lies in no coarse cell");
  Csr P;
  P.nrows = nrows;
  P.ncols = coarse.nfree;
  P.rp.assign(nrows + 1, 0);
  for (int64_t i = 0; i < nrows; ++i) P.rp[i + 1] = P.rp[i] + cnt[i];
  P.ci.resize(P.rp[nrows]);
  P.v.resize(P.rp[nrows]);
  for (int64_t i = 0; i < nrows; ++i)
    for (int k = 0; k < cnt[i]; ++k) P.ci[P.rp[i] + k] = tc[i * nloc + k], P.v[P.rp[i] + k] = tv[i * nloc + k];
  return P;
}

Csr unit_diagonal_on_empty_rows(const Csr& A) {
  // rows with no entries get A_ii = 1 (coarse DoFs that the prolongation never reaches)
  int64_t add = 0;
  for (int64_t i = 0; i < A.nrows; ++i) add += A.rp[i + 1] == A.rp[i];
  if (add == 0) return A;
  Csr B;
  B.nrows = A.nrows;
  B.ncols = A.ncols;
  B.rp.assign(A.nrows + 1, 0);
  B.ci.reserve(A.nnz() + add);
  B.v.reserve(A.nnz() + add);
  for (int64_t i = 0; i < A.nrows; ++i) {
    if (A.rp[i + 1] == A.rp[i]) {
      B.ci.push_back((int32_t)i);
      B.v.push_back(1.0);
    } else {
      B.ci.insert(B.ci.end(), A.ci.begin() + A.rp[i], A.ci.begin() + A.rp[i + 1]);
      B.v.insert(B.v.end(), A.v.begin() + A.rp[i], A.v.begin() + A.rp[i + 1]);
    }
    B.rp[i + 1] = (int32_t)B.ci.size();
  }
  return B;
}

Csr transpose(const Csr& A) {
  Csr T;
  T.nrows = A.ncols;
  T.ncols = A.nrows;
  T.rp.assign(T.nrows + 1, 0);
  for (int32_t c : A.ci) T.rp[c + 1]++;
  for (int64_t i = 0; i < T.nrows; ++i) T.rp[i + 1] += T.rp[i];
  T.ci.resize(A.nnz());
  T.v.resize(A.nnz());
  std::vector<int32_t> fill(T.rp.begin(), T.rp.end() - 1);
  for (int64_t i = 0; i < A.nrows; ++i)
    for (int32_t k = A.rp[i]; k < A.rp[i + 1]; ++k) {
      int32_t pos = fill[A.ci[k]]++;
      T.ci[pos] = (int32_t)i;
      T.v[pos] = A.v[k];
    }
  return T;
}

// C = A B (Gustavson, one pass): row i accumulates in the order of A's row then B's row
// and stores its columns sorted.
Csr spgemm(const Csr& A, const Csr& B) {
  struct State {
    std::vector<int64_t> mark;
    std::vector<double> acc;
    std::vector<int32_t> cols;
  };
  return csr_from_rows(
      A.nrows, B.ncols, [&] { return State{std::vector<int64_t>(B.ncols, -1), std::vector<double>(B.ncols, 0.0), {}}; },
      [&](State& st, int64_t i, std::vector<int32_t>& ci, std::vector<double>& v) {
        st.cols.clear();
        for (int32_t k = A.rp[i]; k < A.rp[i + 1]; ++k) {
          const int32_t r = A.ci[k];
          const double a = A.v[k];
          for (int32_t q = B.rp[r]; q < B.rp[r + 1]; ++q) {
            const int32_t j = B.ci[q];
            if (st.mark[j] != i) {
              st.mark[j] = i;
              st.acc[j] = 0.0;
              st.cols.push_back(j);
            }
            st.acc[j] += a * B.v[q];
          }
        }
        std::sort(st.cols.begin(), st.cols.end());
        for (int32_t j : st.cols) ci.push_back(j), v.push_back(st.acc[j]);
      });
}

std::vector<double> dense_submatrix(const Csr& A, const int32_t* idx, int64_t n) {
  std::vector<double> D((size_t)n * n, 0.0);
  for (int64_t a = 0; a < n; ++a) {
    int32_t r = idx[a];
    for (int32_t k = A.rp[r]; k < A.rp[r + 1]; ++k) {
      const int32_t* p = std::lower_bound(idx, idx + n, A.ci[k]);
      if (p != idx + n && *p == A.ci[k]) D[a * n + (p - idx)] = A.v[k];
    }
  }
  return D;
}

void spmv_host(const Csr& A, const double* x, double* y) {
  parallel_for(A.nrows, [&](int64_t lo, int64_t hi) {
    for (int64_t i = lo; i < hi; ++i) {
      double s = 0;
      for (int32_t k = A.rp[i]; k < A.rp[i + 1]; ++k) s += A.v[k] * x[A.ci[k]];
      y[i] = s;
    }
  });
}

// Number of eigenvalues of the symmetric tridiagonal (a, b) smaller than x (Sturm count).
static int sturm_count(const std::vector<double>& a, const std::vector<double>& b, int m, double x) {
  int c = 0;
  double q = 1.0;
  for (int i = 0; i < m; ++i) {
    double bb = i > 0 ? b[i] * b[i] : 0.0;
    q = a[i] - x - (i > 0 ? bb / q : 0.0);
    if (q == 0.0) q = -1e-300;
    if (q < 0) ++c;
  }
  return c;
}

// Largest eigenvalue of T_m and |last component| of its unit eigenvector.
void tridiag_top(const std::vector<double>& a, const std::vector<double>& b, int m, double* theta, double* slast) {
  double lo = std::numeric_limits<double>::max(), hi = -lo;
  for (int i = 0; i < m; ++i) {
    double r = (i > 0 ? std::fabs(b[i]) : 0.0) + (i + 1 < m ? std::fabs(b[i + 1]) : 0.0);
    lo = std::min(lo, a[i] - r);
    hi = std::max(hi, a[i] + r);
  }
  for (int it = 0; it < 200 && hi - lo > 1e-15 * std::max(1.0, std::fabs(hi)); ++it) {
    double mid = 0.5 * (lo + hi);
    if (sturm_count(a, b, m, mid) == m) hi = mid; else lo = mid;
  }
  *theta = hi;
  // inverse iteration on (T - mu I) with mu just above theta (Thomas algorithm)
  double mu = hi + 1e-10 * std::max(1.0, std::fabs(hi));
  std::vector<double> x(m, 1.0), cp(m), dp(m);
  for (int rep = 0; rep < 3; ++rep) {
    double prev_c = 0;
    for (int i = 0; i < m; ++i) {
      double diag = a[i] - mu - (i > 0 ? b[i] * prev_c : 0.0);
      if (diag == 0.0) diag = 1e-300;
      double up = (i + 1 < m) ? b[i + 1] : 0.0;
      cp[i] = up / diag;
      dp[i] = (x[i] - (i > 0 ? b[i] * dp[i - 1] : 0.0)) / diag;
      prev_c = cp[i];
    }
    for (int i = m - 1; i >= 0; --i) x[i] = dp[i] - (i + 1 < m ? cp[i] * x[i + 1] : 0.0);
    double nrm = 0;
    for (double v : x) nrm += v * v;
    nrm = std::sqrt(nrm);
    for (double& v : x) v /= nrm;
  }
  *slast = std::fabs(x[m - 1]);
}


std::vector<double> lanczos_scaling(const Csr& A, const uint8_t* keep) {
  std::vector<double> s(A.nrows);
  for (int64_t i = 0; i < A.nrows; ++i) {
    double dgn = 0;
    for (int32_t k = A.rp[i]; k < A.rp[i + 1]; ++k)
      if (A.ci[k] == i) dgn = A.v[k];
    s[i] = (keep && !keep[i]) ? 0.0 : 1.0 / std::sqrt(dgn);
  }
  return s;
}

std::vector<double> lanczos_start(const std::vector<double>& s) {
  const int64_t n = (int64_t)s.size();
  std::vector<double> v(n);
  double nrm = 0;
  for (int64_t i = 0; i < n; ++i) {
    uint64_t z = (uint64_t)i * 0x9E3779B97F4A7C15ull + 0x1234567ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    v[i] = s[i] != 0.0 ? (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0 : 0.0;
    nrm += v[i] * v[i];
  }
  nrm = std::sqrt(nrm);
  if (nrm > 0)
    for (auto& x : v) x /= nrm;
  return v;
}

double lanczos_lmax(const Csr& A, const uint8_t* keep, double tol, int maxit, int* iters) {
  const int64_t n = A.nrows;
  std::vector<double> s = lanczos_scaling(A, keep);
  int64_t nk = 0;
  for (int64_t i = 0; i < n; ++i) nk += s[i] != 0.0;
  if (nk == 0) {
    if (iters) *iters = 0;
    return 0.0;
  }
  // deterministic start vector (splitmix64 of the index)
  std::vector<double> v = lanczos_start(s), vprev(n, 0.0), w(n), t(n);
  std::vector<double> al, be(1, 0.0);
  double theta = 0;
  int k = 0;
  for (k = 0; k < std::min<int64_t>(maxit, nk); ++k) {
    for (int64_t i = 0; i < n; ++i) t[i] = s[i] * v[i];
    spmv_host(A, t.data(), w.data());
    double alpha = 0;
    for (int64_t i = 0; i < n; ++i) {
      w[i] *= s[i];
      alpha += w[i] * v[i];
    }
    double beta = 0;
    for (int64_t i = 0; i < n; ++i) {
      w[i] -= alpha * v[i] + be[k] * vprev[i];
      beta += w[i] * w[i];
    }
    beta = std::sqrt(beta);
    al.push_back(alpha);
    be.push_back(beta);
    double sl;
    tridiag_top(al, be, k + 1, &theta, &sl);
    if (beta * sl <= tol * std::fabs(theta) || beta <= 1e-14 * std::fabs(theta)) {
      ++k;
      break;
    }
    for (int64_t i = 0; i < n; ++i) {
      vprev[i] = v[i];
      v[i] = w[i] / beta;
    }
  }
  if (iters) *iters = k;
  return theta;
}

}  // namespace nnmg

namespace nnmg {

// Reverse Cuthill-McKee order of the graph of A (symmetric pattern): breadth-first search
// from a pseudo-peripheral vertex of each connected component, neighbours visited by
// increasing degree, then reversed. Returns perm with perm[new] = old.
std::vector<int32_t> rcm_order(const Csr& A) {
  const int64_t n = A.nrows;
  std::vector<int32_t> deg(n), order;
  order.reserve(n);
  for (int64_t i = 0; i < n; ++i) deg[i] = A.rp[i + 1] - A.rp[i];
  std::vector<uint8_t> seen(n, 0);
  std::vector<int32_t> level(n, -1), nb;
  // breadth-first levels from s inside the unvisited part; returns the last vertex reached
  auto bfs_far = [&](int32_t s, std::vector<int32_t>& visited) {
    visited.clear();
    visited.push_back(s);
    level[s] = 0;
    int32_t far = s;
    for (size_t h = 0; h < visited.size(); ++h) {
      int32_t u = visited[h];
      for (int32_t k = A.rp[u]; k < A.rp[u + 1]; ++k) {
        int32_t w = A.ci[k];
        if (w == u || seen[w] || level[w] >= 0) continue;
        level[w] = level[u] + 1;
        visited.push_back(w);
        if (level[w] > level[far] || (level[w] == level[far] && deg[w] < deg[far])) far = w;
      }
    }
    for (int32_t u : visited) level[u] = -1;
    return far;
  };
  std::vector<int32_t> comp;
  for (int64_t s0 = 0; s0 < n; ++s0) {
    if (seen[s0]) continue;
    int32_t start = (int32_t)s0;
    for (int pass = 0; pass < 2; ++pass) start = bfs_far(start, comp);
    // Cuthill-McKee from `start`
    size_t head = order.size();
    order.push_back(start);
    seen[start] = 1;
    for (size_t h = head; h < order.size(); ++h) {
      int32_t u = order[h];
      nb.clear();
      for (int32_t k = A.rp[u]; k < A.rp[u + 1]; ++k) {
        int32_t w = A.ci[k];
        if (!seen[w]) {
          seen[w] = 1;
          nb.push_back(w);
        }
      }
      std::stable_sort(nb.begin(), nb.end(), [&](int32_t a, int32_t b) { return deg[a] < deg[b]; });
      order.insert(order.end(), nb.begin(), nb.end());
    }
  }
  std::reverse(order.begin(), order.end());
  return order;
}

// B[i, :] = A[rowperm[i], :] with columns renumbered by colmap (old -> new), sorted.
Csr permute_csr(const Csr& A, const std::vector<int32_t>& rowperm, const std::vector<int32_t>& colmap) {
  Csr B;
  B.nrows = A.nrows;
  B.ncols = A.ncols;
  B.rp.assign(A.nrows + 1, 0);
  for (int64_t i = 0; i < A.nrows; ++i) {
    int32_t r = rowperm.empty() ? (int32_t)i : rowperm[i];
    B.rp[i + 1] = B.rp[i] + (A.rp[r + 1] - A.rp[r]);
  }
  B.ci.resize(A.nnz());
  B.v.resize(A.nnz());
  parallel_for(A.nrows, [&](int64_t lo, int64_t hi) {
    std::vector<std::pair<int32_t, double>> row;
    for (int64_t i = lo; i < hi; ++i) {
      int32_t r = rowperm.empty() ? (int32_t)i : rowperm[i];
      row.clear();
      for (int32_t k = A.rp[r]; k < A.rp[r + 1]; ++k)
        row.emplace_back(colmap.empty() ? A.ci[k] : colmap[A.ci[k]], A.v[k]);
      std::sort(row.begin(), row.end(), [](const std::pair<int32_t, double>& a, const std::pair<int32_t, double>& b) {
        return a.first < b.first;
      });
      for (size_t k = 0; k < row.size(); ++k) B.ci[B.rp[i] + k] = row[k].first, B.v[B.rp[i] + k] = row[k].second;
    }
  });
  return B;
}

std::vector<int32_t> inverse_perm(const std::vector<int32_t>& p) {
  std::vector<int32_t> q(p.size());
  for (size_t i = 0; i < p.size(); ++i) q[p[i]] = (int32_t)i;
  return q;
}

int32_t greedy_colouring(const Csr& A, std::vector<int32_t>& colour) {
  const int64_t n = A.nrows;
  std::vector<double> d(n, 0.0);
  for (int64_t i = 0; i < n; ++i)
    for (int32_t k = A.rp[i]; k < A.rp[i + 1]; ++k)
      if (A.ci[k] == i) d[i] = std::sqrt(std::fabs(A.v[k]));
  colour.assign(n, -1);
  std::vector<int64_t> seen;   // seen[c] == i: colour c is held by a neighbour of row i
  int32_t ncol = 0;
  for (int64_t i = 0; i < n; ++i) {
    for (int32_t k = A.rp[i]; k < A.rp[i + 1]; ++k) {
      const int32_t j = A.ci[k];
      if (j == i || colour[j] < 0 || !(std::fabs(A.v[k]) > 1e-12 * d[i] * d[j])) continue;
      if ((size_t)colour[j] >= seen.size()) seen.resize(colour[j] + 1, -1);
      seen[colour[j]] = i;
    }
    int32_t c = 0;
    while ((size_t)c < seen.size() && seen[c] == i) ++c;
    colour[i] = c;
    ncol = std::max(ncol, c + 1);
  }
  return ncol;
}

std::vector<int32_t> morton_order(const std::vector<double>& pts, int dim) {
  const int64_t n = dim > 0 ? (int64_t)pts.size() / dim : 0;
  const int bits = dim == 3 ? 21 : 31;
  double lo[3] = {0, 0, 0}, ext = 0;
  for (int d = 0; d < dim; ++d) {
    double mn = INFINITY, mx = -INFINITY;
    for (int64_t i = 0; i < n; ++i) mn = std::min(mn, pts[i * dim + d]), mx = std::max(mx, pts[i * dim + d]);
    lo[d] = mn;
    ext = std::max(ext, mx - mn);
  }
  const double scale = ext > 0 ? (double)((1u << bits) - 1) / ext : 0.0;
  std::vector<uint64_t> code(n, 0);
  for (int64_t i = 0; i < n; ++i) {
    uint64_t c = 0;
    for (int d = 0; d < dim; ++d) {
      const uint64_t q = (uint64_t)((pts[i * dim + d] - lo[d]) * scale);
      for (int b = 0; b < bits; ++b) c |= ((q >> b) & 1u) << (b * dim + d);
    }
    code[i] = c;
  }
  std::vector<int32_t> ord(n);
  for (int64_t i = 0; i < n; ++i) ord[i] = (int32_t)i;
  std::stable_sort(ord.begin(), ord.end(), [&](int32_t a, int32_t b) { return code[a] < code[b]; });
  return ord;
}

Csr kron_identity(const Csr& P, int d) {
  Csr K;
  K.nrows = P.nrows * d;
  K.ncols = P.ncols * d;
  K.rp.assign(K.nrows + 1, 0);
  for (int64_t i = 0; i < P.nrows; ++i)
    for (int c = 0; c < d; ++c) K.rp[i * d + c + 1] = K.rp[i * d + c] + (P.rp[i + 1] - P.rp[i]);
  K.ci.resize(K.rp[K.nrows]);
  K.v.resize(K.rp[K.nrows]);
  for (int64_t i = 0; i < P.nrows; ++i)
    for (int c = 0; c < d; ++c) {
      int64_t o = K.rp[i * d + c];
      for (int32_t k = P.rp[i]; k < P.rp[i + 1]; ++k, ++o) K.ci[o] = P.ci[k] * d + c, K.v[o] = P.v[k];
    }
  return K;
}

}  // namespace nnmg
