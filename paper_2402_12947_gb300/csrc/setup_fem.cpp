// Host set-up, part 1: DoF maps, Poisson stiffness, cell quality and local patches.
//
// Discretisation as in Sec. 2 / Sec. 6.1 of Chen & Wells (continuous Lagrange P1/P2 on
// simplices, Dirichlet DoFs eliminated with g = 0). Element integrals are evaluated in
// closed form: every P2 basis gradient is a combination sum_p c_p(lambda) grad(lambda_p)
// with c_p affine in the barycentric coordinates, and products of two affine functions
// integrate exactly with int_K lambda_r = |K|/(d+1) and
// int_K lambda_r lambda_s = |K| d! (1 + delta_rs) / (d+2)!.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <thread>

#include "internal.hpp"

namespace nnmg {

namespace {
thread_local int tl_thread_budget = 0;
}

void set_thread_budget(int k) { tl_thread_budget = k; }

int num_threads() {
  unsigned n = std::thread::hardware_concurrency();
  int all = (int)std::max(1u, std::min(n, 32u));
  return tl_thread_budget > 0 ? std::min(all, tl_thread_budget) : all;
}

void parallel_for(int64_t n, const std::function<void(int64_t, int64_t)>& body) {
  int nt = num_threads();
  if (n < 4096 || nt == 1) {
    body(0, n);
    return;
  }
  std::vector<std::thread> th;
  int64_t chunk = (n + nt - 1) / nt;
  for (int t = 0; t < nt; ++t) {
    int64_t lo = t * chunk, hi = std::min(n, lo + chunk);
    if (lo >= hi) break;
    th.emplace_back(body, lo, hi);
  }
  for (auto& t : th) t.join();
}

namespace {

// Groups k-tuples (each sorted ascending) by lexicographic order. Returns the number of
// distinct tuples; id[i] is the rank of tuple i among the distinct ones, mult[u] the
// multiplicity of distinct tuple u and first[u] the index of one tuple equal to it.
struct TupleGroups {
  int64_t nuniq = 0;
  std::vector<int64_t> id, first;
  std::vector<int32_t> mult;
};

TupleGroups group_tuples(const std::vector<int64_t>& t, int k, int64_t nv) {
  int64_t n = (int64_t)t.size() / k;
  std::vector<int64_t> start(nv + 1, 0);
  for (int64_t i = 0; i < n; ++i) start[t[i * k] + 1]++;
  for (int64_t v = 0; v < nv; ++v) start[v + 1] += start[v];
  std::vector<int64_t> order(n), fill(start.begin(), start.end() - 1);
  for (int64_t i = 0; i < n; ++i) order[fill[t[i * k]]++] = i;
  auto less = [&](int64_t a, int64_t b) {
    for (int j = 1; j < k; ++j)
      if (t[a * k + j] != t[b * k + j]) return t[a * k + j] < t[b * k + j];
    return false;
  };
  auto equal = [&](int64_t a, int64_t b) {
    for (int j = 0; j < k; ++j)
      if (t[a * k + j] != t[b * k + j]) return false;
    return true;
  };
  parallel_for(nv, [&](int64_t lo, int64_t hi) {
    for (int64_t v = lo; v < hi; ++v)
      std::sort(order.begin() + start[v], order.begin() + start[v + 1], less);
  });
  TupleGroups g;
  g.id.assign(n, -1);
  for (int64_t i = 0; i < n; ++i) {
    int64_t cur = order[i];
    if (i == 0 || !equal(order[i - 1], cur)) {
      g.first.push_back(cur);
      g.mult.push_back(0);
    }
    g.id[cur] = (int64_t)g.first.size() - 1;
    g.mult.back()++;
  }
  g.nuniq = (int64_t)g.first.size();
  return g;
}

const int kEdges2[3][2] = {{0, 1}, {0, 2}, {1, 2}};
const int kEdges3[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};

inline const int (*local_edges(int dim))[2] { return dim == 2 ? kEdges2 : kEdges3; }
inline int num_local_edges(int dim) { return dim == 2 ? 3 : 6; }

// Barycentric gradients G[(d+1)*d] and |K| of one cell.
bool cell_geometry(const MeshH& m, int64_t c, double* G, double* vol) {
  const int d = m.dim;
  const int32_t* cv = &m.c[c * (d + 1)];
  const double* x0 = &m.x[(int64_t)cv[0] * d];
  double J[3][3];
  for (int i = 0; i < d; ++i)
    for (int r = 0; r < d; ++r) J[r][i] = m.x[(int64_t)cv[i + 1] * d + r] - x0[r];
  double Ji[3][3], det;
  if (d == 2) {
    det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    if (det == 0.0) return false;
    Ji[0][0] = J[1][1] / det;  Ji[0][1] = -J[0][1] / det;
    Ji[1][0] = -J[1][0] / det; Ji[1][1] = J[0][0] / det;
    *vol = std::fabs(det) / 2.0;
  } else {
    double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
    if (det == 0.0) return false;
    Ji[0][0] = c00 / det;
    Ji[1][0] = c01 / det;
    Ji[2][0] = c02 / det;
    Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
    Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
    Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
    Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
    Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
    Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
    *vol = std::fabs(det) / 6.0;
  }
  // grad lambda_p (p >= 1) is row p-1 of J^{-1}; grad lambda_0 = -sum of the others
  for (int r = 0; r < d; ++r) {
    double s = 0;
    for (int p = 1; p <= d; ++p) {
      G[p * d + r] = Ji[p - 1][r];
      s += Ji[p - 1][r];
    }
    G[r] = -s;
  }
  return true;
}

// Affine coefficient functions of a basis gradient: grad phi = sum_t c_t(lambda) G_{p_t}.
struct Affine {
  double c0;
  double c[4];
};
struct GradTerm {
  int nterms;
  int p[2];
  Affine f[2];
};

GradTerm basis_term(int degree, int dim, int a) {
  GradTerm g{};
  if (degree == 1) {
    g.nterms = 1;
    g.p[0] = a;
    g.f[0].c0 = 1.0;
    return g;
  }
  if (a <= dim) {
    g.nterms = 1;
    g.p[0] = a;
    g.f[0].c0 = -1.0;
    g.f[0].c[a] = 4.0;
    return g;
  }
  const int(*le)[2] = local_edges(dim);
  int s = le[a - dim - 1][0], t = le[a - dim - 1][1];
  g.nterms = 2;
  g.p[0] = s;
  g.f[0].c[t] = 4.0;
  g.p[1] = t;
  g.f[1].c[s] = 4.0;
  return g;
}

double factorial(int n) { return n <= 1 ? 1.0 : n * factorial(n - 1); }

// int_K f g / |K| for affine f, g.
double affine_product_mean(const Affine& f, const Affine& g, int d) {
  const double m1 = 1.0 / (d + 1);
  const double m2 = factorial(d) / factorial(d + 2);
  double s = f.c0 * g.c0;
  double sf = 0, sg = 0;
  for (int r = 0; r <= d; ++r) {
    sf += f.c[r];
    sg += g.c[r];
  }
  s += (f.c0 * sg + g.c0 * sf) * m1;
  double q = 0;
  for (int r = 0; r <= d; ++r)
    for (int t = 0; t <= d; ++t) q += f.c[r] * g.c[t] * (r == t ? 2.0 : 1.0);
  return s + q * m2;
}

}  // namespace

DofMapH build_dofmap(const MeshH& m, int degree) {
  DofMapH dm;
  const int d = m.dim, d1 = d + 1;
  dm.degree = degree;
  dm.dim = d;
  dm.nv = m.nv;
  // boundary facets: facets (sorted vertex tuples) that belong to exactly one cell
  std::vector<int64_t> fac((size_t)m.nc * d1 * d);
  parallel_for(m.nc, [&](int64_t lo, int64_t hi) {
    for (int64_t c = lo; c < hi; ++c)
      for (int i = 0; i < d1; ++i) {
        int64_t tmp[3];
        int k = 0;
        for (int j = 0; j < d1; ++j)
          if (j != i) tmp[k++] = m.c[c * d1 + j];
        std::sort(tmp, tmp + d);
        for (int j = 0; j < d; ++j) fac[(c * d1 + i) * d + j] = tmp[j];
      }
  });
  TupleGroups fg = group_tuples(fac, d, m.nv);
  std::vector<uint8_t> vdir(m.nv, 0);
  std::vector<int64_t> bfacets;  // first-occurrence index of each boundary facet
  for (int64_t u = 0; u < fg.nuniq; ++u)
    if (fg.mult[u] == 1) {
      int64_t f = fg.first[u];
      bfacets.push_back(f);
      for (int j = 0; j < d; ++j) {
        int64_t v = fac[f * d + j];
        if (m.mask.empty() || m.mask[v]) vdir[v] = 1;
      }
    }
  dm.bfaces = bfacets;
  fac.clear();
  fac.shrink_to_fit();
  std::vector<int64_t> facets_kept;  // vertex tuples of boundary facets
  // (recomputed below only when P2 needs them)
  if (degree == 1) {
    dm.nloc = d1;
    dm.ndofs = m.nv;
    dm.cell_dofs.assign(m.c.begin(), m.c.end());
    dm.points = m.x;
    dm.dirichlet = vdir;
  } else {
    const int ne = num_local_edges(d);
    const int(*le)[2] = local_edges(d);
    dm.nloc = d1 + ne;
    std::vector<int64_t> et((size_t)m.nc * ne * 2);
    parallel_for(m.nc, [&](int64_t lo, int64_t hi) {
      for (int64_t c = lo; c < hi; ++c)
        for (int e = 0; e < ne; ++e) {
          int64_t a = m.c[c * d1 + le[e][0]], b = m.c[c * d1 + le[e][1]];
          et[(c * ne + e) * 2] = std::min(a, b);
          et[(c * ne + e) * 2 + 1] = std::max(a, b);
        }
    });
    TupleGroups eg = group_tuples(et, 2, m.nv);
    int64_t nedges = eg.nuniq;
    dm.edges.resize(nedges * 2);
    for (int64_t u = 0; u < nedges; ++u) {
      dm.edges[u * 2] = et[eg.first[u] * 2];
      dm.edges[u * 2 + 1] = et[eg.first[u] * 2 + 1];
    }
    dm.ndofs = m.nv + nedges;
    dm.cell_dofs.resize((size_t)m.nc * dm.nloc);
    parallel_for(m.nc, [&](int64_t lo, int64_t hi) {
      for (int64_t c = lo; c < hi; ++c) {
        for (int i = 0; i < d1; ++i) dm.cell_dofs[c * dm.nloc + i] = m.c[c * d1 + i];
        for (int e = 0; e < ne; ++e) dm.cell_dofs[c * dm.nloc + d1 + e] = m.nv + eg.id[c * ne + e];
      }
    });
    dm.points.resize(dm.ndofs * d);
    std::copy(m.x.begin(), m.x.end(), dm.points.begin());
    for (int64_t u = 0; u < nedges; ++u)
      for (int r = 0; r < d; ++r)
        dm.points[(m.nv + u) * d + r] = 0.5 * (m.x[dm.edges[u * 2] * d + r] + m.x[dm.edges[u * 2 + 1] * d + r]);
    // edge lookup: edges starting at vertex a are contiguous and sorted by their end
    std::vector<int64_t> estart(m.nv + 1, 0);
    for (int64_t u = 0; u < nedges; ++u) estart[dm.edges[u * 2] + 1]++;
    for (int64_t v = 0; v < m.nv; ++v) estart[v + 1] += estart[v];
    auto edge_id = [&](int64_t a, int64_t b) -> int64_t {
      if (a > b) std::swap(a, b);
      int64_t lo = estart[a], hi = estart[a + 1];
      while (lo < hi) {
        int64_t mid = (lo + hi) / 2;
        if (dm.edges[mid * 2 + 1] < b) lo = mid + 1; else hi = mid;
      }
      return (lo < estart[a + 1] && dm.edges[lo * 2 + 1] == b) ? lo : -1;
    };
    dm.dirichlet.assign(dm.ndofs, 0);
    std::copy(vdir.begin(), vdir.end(), dm.dirichlet.begin());
    // an edge DoF is Dirichlet if its edge lies in a boundary facet and both ends are
    for (int64_t f : bfacets) {
      int64_t c = f / d1, i = f % d1;
      int64_t vs[3];
      int k = 0;
      for (int j = 0; j < d1; ++j)
        if (j != i) vs[k++] = m.c[c * d1 + j];
      for (int a = 0; a < d; ++a)
        for (int b = a + 1; b < d; ++b) {
          if (!vdir[vs[a]] || !vdir[vs[b]]) continue;
          int64_t e = edge_id(vs[a], vs[b]);
          if (e >= 0) dm.dirichlet[m.nv + e] = 1;
        }
    }
  }
  dm.free_index.assign(dm.ndofs, -1);
  for (int64_t i = 0; i < dm.ndofs; ++i)
    if (!dm.dirichlet[i]) {
      dm.free_index[i] = (int64_t)dm.free_list.size();
      dm.free_list.push_back(i);
    }
  dm.nfree = (int64_t)dm.free_list.size();
  return dm;
}

std::vector<double> radius_ratio(const MeshH& m) {
  const int d = m.dim, d1 = d + 1;
  std::vector<double> g(m.nc);
  parallel_for(m.nc, [&](int64_t lo, int64_t hi) {
    for (int64_t c = lo; c < hi; ++c) {
      const int32_t* cv = &m.c[c * d1];
      auto X = [&](int i, int r) { return m.x[(int64_t)cv[i] * d + r]; };
      if (d == 2) {
        double ex[3], ey[3], len[3];
        for (int i = 0; i < 3; ++i) {
          int a = (i + 1) % 3, b = (i + 2) % 3;
          ex[i] = X(b, 0) - X(a, 0);
          ey[i] = X(b, 1) - X(a, 1);
          len[i] = std::sqrt(ex[i] * ex[i] + ey[i] * ey[i]);
        }
        double area = 0.5 * std::fabs(ex[2] * ey[0] - ey[2] * ex[0]);
        // R_I = area / semi-perimeter; R_C = abc / (4 area)
        double rin = area / (0.5 * (len[0] + len[1] + len[2]));
        double rc = len[0] * len[1] * len[2] / (4.0 * area);
        g[c] = (area > 0) ? 2.0 * rin / rc : 0.0;
      } else {
        double a[3], b[3], e[3];
        for (int r = 0; r < 3; ++r) {
          a[r] = X(1, r) - X(0, r);
          b[r] = X(2, r) - X(0, r);
          e[r] = X(3, r) - X(0, r);
        }
        auto cross = [](const double* u, const double* v, double* w) {
          w[0] = u[1] * v[2] - u[2] * v[1];
          w[1] = u[2] * v[0] - u[0] * v[2];
          w[2] = u[0] * v[1] - u[1] * v[0];
        };
        auto dot = [](const double* u, const double* v) { return u[0] * v[0] + u[1] * v[1] + u[2] * v[2]; };
        double bxe[3], exa[3], axb[3];
        cross(b, e, bxe);
        cross(e, a, exa);
        cross(a, b, axb);
        double six_v = dot(a, bxe);
        double vol = std::fabs(six_v) / 6.0;
        // circumcentre offset from v0: (|a|^2 b x e + |b|^2 e x a + |e|^2 a x b) / (2 a.(b x e))
        double aa = dot(a, a), bb = dot(b, b), ee = dot(e, e), w[3];
        for (int r = 0; r < 3; ++r) w[r] = (aa * bxe[r] + bb * exa[r] + ee * axb[r]) / (2.0 * six_v);
        double rc = std::sqrt(dot(w, w));
        // face areas: |a x b|/2 (v0v1v2), |b x e|/2 (v0v2v3), |e x a|/2 (v0v3v1), and v1v2v3
        double u1[3], u2[3], n4[3];
        for (int r = 0; r < 3; ++r) {
          u1[r] = b[r] - a[r];
          u2[r] = e[r] - a[r];
        }
        cross(u1, u2, n4);
        double S = 0.5 * (std::sqrt(dot(axb, axb)) + std::sqrt(dot(bxe, bxe)) + std::sqrt(dot(exa, exa)) +
                          std::sqrt(dot(n4, n4)));
        double rin = 3.0 * vol / S;
        g[c] = (vol > 0) ? 3.0 * rin / rc : 0.0;
      }
    }
  });
  return g;
}

Csr assemble_stiffness(const MeshH& m, const DofMapH& dm) {
  const int d = m.dim, d1 = d + 1, nloc = dm.nloc;
  // DoF -> cells incidence (cells ascending per DoF)
  std::vector<int64_t> dstart(dm.ndofs + 1, 0);
  for (int64_t k = 0; k < m.nc * nloc; ++k) dstart[dm.cell_dofs[k] + 1]++;
  for (int64_t i = 0; i < dm.ndofs; ++i) dstart[i + 1] += dstart[i];
  std::vector<int64_t> dcells(dstart[dm.ndofs]), fill(dstart.begin(), dstart.end() - 1);
  std::vector<int8_t> dlocal(dstart[dm.ndofs]);
  for (int64_t c = 0; c < m.nc; ++c)
    for (int a = 0; a < nloc; ++a) {
      int64_t g = dm.cell_dofs[c * nloc + a];
      dlocal[fill[g]] = (int8_t)a;
      dcells[fill[g]++] = c;
    }
  // per cell: |K| and the Gram matrix G G^T of the barycentric gradients (rows of G), computed
  // once instead of once per row of the cell; degenerate cells are an error (the first one)
  std::vector<double> cvol(m.nc), cgg((size_t)m.nc * d1 * d1);
  std::vector<uint8_t> bad(m.nc, 0);
  parallel_for(m.nc, [&](int64_t lo, int64_t hi) {
    for (int64_t c = lo; c < hi; ++c) {
      double G[12], vol;
      if (!cell_geometry(m, c, G, &vol) || !(vol > 0)) {
        bad[c] = 1;
        continue;
      }
      cvol[c] = vol;
      double* gg = &cgg[(size_t)c * d1 * d1];
      for (int p = 0; p < d1; ++p)
        for (int q = 0; q < d1; ++q) {
          double s = 0;
          for (int r = 0; r < d; ++r) s += G[p * d + r] * G[q * d + r];
          gg[p * d1 + q] = s;
        }
    }
  });
  for (int64_t c = 0; c < m.nc; ++c)
    if (bad[c]) throw Error(MG_ERR_DEGENERATE_CELL, "cell " + std::to_string(c) + " has zero volume");
  GradTerm terms[10];
  for (int a = 0; a < nloc; ++a) terms[a] = basis_term(dm.degree, d, a);
  // the means of the products of the basis gradients' affine factors, per (a, s, b, t)
  double pm[10][2][10][2];
  for (int a = 0; a < nloc; ++a)
    for (int s = 0; s < terms[a].nterms; ++s)
      for (int b = 0; b < nloc; ++b)
        for (int t = 0; t < terms[b].nterms; ++t) pm[a][s][b][t] = affine_product_mean(terms[a].f[s], terms[b].f[t], d);
  // one pass per row: its pattern (free columns sharing a cell, sorted), then its values,
  // summed over its cells in ascending cell order
  return csr_from_rows(
      dm.nfree, dm.nfree, [] { return std::vector<int32_t>(); },
      [&](std::vector<int32_t>& buf, int64_t i, std::vector<int32_t>& ci, std::vector<double>& v) {
        const int64_t g = dm.free_list[i];
        buf.clear();
        for (int64_t k = dstart[g]; k < dstart[g + 1]; ++k) {
          const int64_t c = dcells[k];
          for (int b = 0; b < nloc; ++b) {
            const int64_t fj = dm.free_index[dm.cell_dofs[c * nloc + b]];
            if (fj >= 0) buf.push_back((int32_t)fj);
          }
        }
        std::sort(buf.begin(), buf.end());
        buf.erase(std::unique(buf.begin(), buf.end()), buf.end());
        const size_t r0 = ci.size();
        ci.insert(ci.end(), buf.begin(), buf.end());
        v.resize(ci.size(), 0.0);
        const int32_t* rc = ci.data() + r0;
        double* rv = v.data() + r0;
        for (int64_t k = dstart[g]; k < dstart[g + 1]; ++k) {
          const int64_t c = dcells[k];
          const int a = dlocal[k];
          const double vol = cvol[c];
          const double* gg = &cgg[(size_t)c * d1 * d1];
          for (int b = 0; b < nloc; ++b) {
            const int64_t fj = dm.free_index[dm.cell_dofs[c * nloc + b]];
            if (fj < 0) continue;
            double kab = 0;
            for (int s = 0; s < terms[a].nterms; ++s)
              for (int t = 0; t < terms[b].nterms; ++t) kab += gg[terms[a].p[s] * d1 + terms[b].p[t]] * pm[a][s][b][t];
            const int64_t pos = std::lower_bound(rc, rc + buf.size(), (int32_t)fj) - rc;
            rv[pos] += vol * kab;
          }
        }
      });
}

std::vector<double> load_constant(const MeshH& m, const DofMapH& dm, double f) {
  const int d = m.dim, nloc = dm.nloc;
  // int_K phi_a / |K|: P1 1/(d+1); P2 vertex 2*2 d!/(d+2)! - 1/(d+1), edge 4 d!/(d+2)!
  double wv, we = 0.0;
  if (dm.degree == 1) {
    wv = 1.0 / (d + 1);
  } else {
    double m2 = factorial(d) / factorial(d + 2);
    wv = 4.0 * m2 - 1.0 / (d + 1);
    we = 4.0 * m2;
  }
  std::vector<double> all(dm.ndofs, 0.0);
  for (int64_t c = 0; c < m.nc; ++c) {
    double G[12], vol;
    if (!cell_geometry(m, c, G, &vol)) throw Error(MG_ERR_DEGENERATE_CELL, "degenerate cell");
    for (int a = 0; a < nloc; ++a) all[dm.cell_dofs[c * nloc + a]] += f * vol * (a <= d ? wv : we);
  }
  std::vector<double> b(dm.nfree);
  for (int64_t i = 0; i < dm.nfree; ++i) b[i] = all[dm.free_list[i]];
  return b;
}

void local_patches(const MeshH& m, const DofMapH& dm, const std::vector<double>& gamma, double threshold,
                   int layers, std::vector<int32_t>& ptr, std::vector<int32_t>& dofs) {
  const int d1 = m.dim + 1;
  ptr.assign(1, 0);
  dofs.clear();
  std::vector<uint8_t> region(m.nc, 0);
  bool any = false;
  for (int64_t c = 0; c < m.nc; ++c)
    if (gamma[c] < threshold) region[c] = 1, any = true;
  if (!any) return;
  for (int l = 0; l < layers; ++l) {
    std::vector<uint8_t> vmark(m.nv, 0);
    for (int64_t c = 0; c < m.nc; ++c)
      if (region[c])
        for (int j = 0; j < d1; ++j) vmark[m.c[c * d1 + j]] = 1;
    for (int64_t c = 0; c < m.nc; ++c)
      if (!region[c])
        for (int j = 0; j < d1; ++j)
          if (vmark[m.c[c * d1 + j]]) {
            region[c] = 1;
            break;
          }
  }
  // union-find over vertices: the cells of one component share vertices transitively
  std::vector<int64_t> parent(m.nv);
  std::iota(parent.begin(), parent.end(), 0);
  std::function<int64_t(int64_t)> find = [&](int64_t v) {
    while (parent[v] != v) {
      parent[v] = parent[parent[v]];
      v = parent[v];
    }
    return v;
  };
  for (int64_t c = 0; c < m.nc; ++c)
    if (region[c])
      for (int j = 1; j < d1; ++j) {
        int64_t a = find(m.c[c * d1]), b = find(m.c[c * d1 + j]);
        if (a != b) parent[std::max(a, b)] = std::min(a, b);
      }
  std::vector<std::pair<int64_t, int32_t>> tagged;  // (component root, free dof)
  for (int64_t c = 0; c < m.nc; ++c)
    if (region[c]) {
      int64_t root = find(m.c[c * d1]);
      for (int a = 0; a < dm.nloc; ++a) {
        int64_t f = dm.free_index[dm.cell_dofs[c * dm.nloc + a]];
        if (f >= 0) tagged.emplace_back(root, (int32_t)f);
      }
    }
  std::sort(tagged.begin(), tagged.end());
  tagged.erase(std::unique(tagged.begin(), tagged.end()), tagged.end());
  std::vector<std::vector<int32_t>> groups;
  for (size_t i = 0; i < tagged.size(); ++i) {
    if (i == 0 || tagged[i].first != tagged[i - 1].first) groups.emplace_back();
    groups.back().push_back(tagged[i].second);
  }
  std::sort(groups.begin(), groups.end(),
            [](const std::vector<int32_t>& a, const std::vector<int32_t>& b) { return a[0] < b[0]; });
  for (auto& g : groups) {
    dofs.insert(dofs.end(), g.begin(), g.end());
    ptr.push_back((int32_t)dofs.size());
  }
}


Csr assemble_elasticity(const MeshH& m, const DofMapH& dm, double mu, double lam) {
  const int d = m.dim, nloc = dm.nloc;
  std::vector<int64_t> dstart(dm.ndofs + 1, 0);
  for (int64_t k = 0; k < m.nc * nloc; ++k) dstart[dm.cell_dofs[k] + 1]++;
  for (int64_t i = 0; i < dm.ndofs; ++i) dstart[i + 1] += dstart[i];
  std::vector<int64_t> dcells(dstart[dm.ndofs]), fill(dstart.begin(), dstart.end() - 1);
  std::vector<int8_t> dlocal(dstart[dm.ndofs]);
  for (int64_t c = 0; c < m.nc; ++c)
    for (int a = 0; a < nloc; ++a) {
      int64_t g = dm.cell_dofs[c * nloc + a];
      dlocal[fill[g]] = (int8_t)a;
      dcells[fill[g]++] = c;
    }
  for (int64_t c = 0; c < m.nc; ++c) {
    double G[12], vol;
    if (!cell_geometry(m, c, G, &vol) || !(vol > 0))
      throw Error(MG_ERR_DEGENERATE_CELL, "cell " + std::to_string(c) + " has zero volume");
  }
  // scalar row patterns (free nodes sharing a cell), then d rows of d * len entries each
  const int64_t nf = dm.nfree;
  std::vector<std::vector<int32_t>> pat(nf);
  parallel_for(nf, [&](int64_t lo, int64_t hi) {
    for (int64_t i = lo; i < hi; ++i) {
      int64_t g = dm.free_list[i];
      std::vector<int32_t>& buf = pat[i];
      for (int64_t k = dstart[g]; k < dstart[g + 1]; ++k) {
        int64_t c = dcells[k];
        for (int b = 0; b < nloc; ++b) {
          int64_t fj = dm.free_index[dm.cell_dofs[c * nloc + b]];
          if (fj >= 0) buf.push_back((int32_t)fj);
        }
      }
      std::sort(buf.begin(), buf.end());
      buf.erase(std::unique(buf.begin(), buf.end()), buf.end());
    }
  });
  Csr A;
  A.nrows = A.ncols = nf * d;
  if (A.nrows > INT32_MAX) throw Error(MG_ERR_INVALID_ARG, "too many vector DoFs");
  A.rp.assign(A.nrows + 1, 0);
  for (int64_t i = 0; i < nf; ++i)
    for (int c = 0; c < d; ++c) {
      const int64_t r = i * d + c;
      if ((int64_t)A.rp[r] + (int64_t)pat[i].size() * d > INT32_MAX) throw Error(MG_ERR_INVALID_ARG, "nnz exceeds 2^31");
      A.rp[r + 1] = A.rp[r] + (int32_t)pat[i].size() * d;
    }
  A.ci.resize(A.rp[A.nrows]);
  A.v.assign(A.rp[A.nrows], 0.0);
  GradTerm terms[10];
  for (int a = 0; a < nloc; ++a) terms[a] = basis_term(dm.degree, d, a);
  double pm[10][2][10][2];   // means of the products of the gradients' affine factors
  for (int a = 0; a < nloc; ++a)
    for (int s1 = 0; s1 < terms[a].nterms; ++s1)
      for (int b = 0; b < nloc; ++b)
        for (int t1 = 0; t1 < terms[b].nterms; ++t1) pm[a][s1][b][t1] = affine_product_mean(terms[a].f[s1], terms[b].f[t1], d);
  parallel_for(nf, [&](int64_t lo, int64_t hi) {
    for (int64_t i = lo; i < hi; ++i) {
      const std::vector<int32_t>& cols = pat[i];
      const int64_t len = (int64_t)cols.size();
      for (int c = 0; c < d; ++c) {
        int32_t* rc = &A.ci[A.rp[i * d + c]];
        for (int64_t q = 0; q < len; ++q)
          for (int e = 0; e < d; ++e) rc[q * d + e] = cols[q] * d + e;
      }
      const int64_t g = dm.free_list[i];
      for (int64_t k = dstart[g]; k < dstart[g + 1]; ++k) {
        const int64_t cell = dcells[k];
        const int a = dlocal[k];
        double G[12], vol;
        cell_geometry(m, cell, G, &vol);
        for (int b = 0; b < nloc; ++b) {
          const int64_t fj = dm.free_index[dm.cell_dofs[cell * nloc + b]];
          if (fj < 0) continue;
          // M[r][s] = int d_r phi_a d_s phi_b / |K|
          double M[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
          for (int s1 = 0; s1 < terms[a].nterms; ++s1)
            for (int t1 = 0; t1 < terms[b].nterms; ++t1) {
              const double w = pm[a][s1][b][t1];
              const double* ga = &G[terms[a].p[s1] * d];
              const double* gb = &G[terms[b].p[t1] * d];
              for (int r = 0; r < d; ++r)
                for (int s2 = 0; s2 < d; ++s2) M[r][s2] += w * ga[r] * gb[s2];
            }
          double S = 0;
          for (int r = 0; r < d; ++r) S += M[r][r];
          const int64_t pos = std::lower_bound(cols.begin(), cols.end(), (int32_t)fj) - cols.begin();
          for (int ci = 0; ci < d; ++ci) {
            double* rv = &A.v[A.rp[i * d + ci] + pos * d];
            for (int cj = 0; cj < d; ++cj)
              rv[cj] += vol * ((ci == cj ? mu * S : 0.0) + mu * M[cj][ci] + lam * M[ci][cj]);
          }
        }
      }
    }
  });
  return A;
}

BoundaryFaces boundary_faces(const MeshH& m, const DofMapH& dm) {
  BoundaryFaces bf;
  const int d = m.dim, d1 = d + 1;
  bf.dim = d;
  bf.degree = dm.degree;
  const int ne = dm.degree == 2 ? (d == 2 ? 1 : 3) : 0;
  bf.nfloc = d + ne;
  const int64_t nf = (int64_t)dm.bfaces.size();
  bf.x.resize(nf * d * d);
  bf.dofs.resize(nf * bf.nfloc);
  for (int64_t f = 0; f < nf; ++f) {
    const int64_t c = dm.bfaces[f] / d1;
    const int opp = (int)(dm.bfaces[f] % d1);
    int k = 0;
    for (int j = 0; j < d1; ++j) {
      if (j == opp) continue;
      const int64_t v = m.c[c * d1 + j];
      for (int r = 0; r < d; ++r) bf.x[(f * d + k) * d + r] = m.x[v * d + r];
      bf.dofs[f * bf.nfloc + k] = dm.free_index[dm.cell_dofs[c * dm.nloc + j]];
      ++k;
    }
    if (ne) {
      const int (*le)[2] = local_edges(d);
      for (int e = 0; e < num_local_edges(d); ++e)
        if (le[e][0] != opp && le[e][1] != opp)
          bf.dofs[f * bf.nfloc + k++] = dm.free_index[dm.cell_dofs[c * dm.nloc + d1 + e]];
    }
  }
  return bf;
}

std::vector<double> traction_load(const BoundaryFaces& bf, int axis, double value, double tol, const double* t,
                                  int64_t nfree) {
  const int d = bf.dim;
  std::vector<double> b(nfree * d, 0.0);
  const int64_t nf = bf.nfloc ? (int64_t)bf.dofs.size() / bf.nfloc : 0;
  for (int64_t f = 0; f < nf; ++f) {
    const double* X = &bf.x[f * d * d];
    bool on = true;
    for (int k = 0; k < d; ++k) on = on && std::fabs(X[k * d + axis] - value) <= tol;
    if (!on) continue;
    // facet measure: segment length (2D) or triangle area (3D)
    double area;
    if (d == 2) {
      area = std::hypot(X[2] - X[0], X[3] - X[1]);
    } else {
      double u[3], w[3];
      for (int r = 0; r < 3; ++r) u[r] = X[3 + r] - X[r], w[r] = X[6 + r] - X[r];
      const double cx = u[1] * w[2] - u[2] * w[1], cy = u[2] * w[0] - u[0] * w[2], cz = u[0] * w[1] - u[1] * w[0];
      area = 0.5 * std::sqrt(cx * cx + cy * cy + cz * cz);
    }
    // int_F phi: P1 |F|/d per vertex; P2 segment |F|/6 (vertex), 2|F|/3 (midpoint);
    // P2 triangle 0 (vertex), |F|/3 (edge)
    double wv, we = 0.0;
    if (bf.degree == 1) wv = area / d;
    else if (d == 2) wv = area / 6.0, we = 2.0 * area / 3.0;
    else wv = 0.0, we = area / 3.0;
    for (int k = 0; k < bf.nfloc; ++k) {
      const int64_t g = bf.dofs[f * bf.nfloc + k];
      if (g < 0) continue;
      const double w = k < d ? wv : we;
      for (int c = 0; c < d; ++c) b[g * d + c] += t[c] * w;
    }
  }
  return b;
}

}  // namespace nnmg
