// Host-side construction of the Taylor-Hood P2/P1 discrete structure:
// P2 numbering, Dirichlet nodes, element geometry, the CSR patterns of the
// shared scalar block F and the divergence block B (Section 2, conforming
// inf-sup stable pair), the element -> nonzero scatter maps that let the
// device assemble without atomics, and the smoothed-aggregation hierarchy of
// the pressure Laplacian used by the block preconditioner.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <numeric>

#include "mhde_internal.h"

namespace mhde {

namespace {

// local edges of a triangle in P2 node order 3, 4, 5
const int LE[3][2] = {{0, 1}, {1, 2}, {2, 0}};

// Sort (key, payload) pairs by key then payload; returns unique keys and, for
// every input, the index of its key in the unique list.
void unique_keys(const std::vector<long long>& keys, std::vector<long long>& uniq,
                 std::vector<int>& where) {
  std::vector<int> order(keys.size());
  std::iota(order.begin(), order.end(), 0);
  std::sort(order.begin(), order.end(), [&](int a, int b) {
    return keys[a] < keys[b] || (keys[a] == keys[b] && a < b);
  });
  uniq.clear();
  where.assign(keys.size(), -1);
  for (size_t t = 0; t < order.size(); ++t) {
    long long k = keys[order[t]];
    if (uniq.empty() || uniq.back() != k) uniq.push_back(k);
    where[order[t]] = (int)uniq.size() - 1;
  }
}

// CSR pattern from sorted unique keys row * ncols + col.
void csr_from_keys(const std::vector<long long>& uniq, int nrows, int ncols, HostCsr& A) {
  A.nrows = nrows;
  A.ncols = ncols;
  A.rowptr.assign(nrows + 1, 0);
  A.col.resize(uniq.size());
  for (size_t k = 0; k < uniq.size(); ++k) {
    int r = (int)(uniq[k] / ncols);
    A.col[k] = (int)(uniq[k] % ncols);
    A.rowptr[r + 1]++;
  }
  for (int r = 0; r < nrows; ++r) A.rowptr[r + 1] += A.rowptr[r];
}

// Inverse of a slot -> nnz map: for every nnz, the slots mapping to it,
// ascending (a fixed summation order).
void invert_map(const std::vector<int>& slot_nnz, long long nnz, std::vector<int>& ptr,
                std::vector<int>& slots) {
  ptr.assign(nnz + 1, 0);
  for (int k : slot_nnz) ptr[k + 1]++;
  for (long long k = 0; k < nnz; ++k) ptr[k + 1] += ptr[k];
  std::vector<int> fill(ptr.begin(), ptr.end() - 1);
  slots.resize(slot_nnz.size());
  for (size_t s = 0; s < slot_nnz.size(); ++s) slots[fill[slot_nnz[s]]++] = (int)s;
}

}  // namespace

std::string build_fe(const mhde_mesh* mesh, FeHost& fe, int element) {
  if (!mesh || !mesh->xy || !mesh->tri) return "mesh pointers are NULL";
  if (element != 0 && element != 1) return "element must be 0 or 1";
  fe.element = element;
  if (mesh->nv < 3 || mesh->nt < 1) return "mesh needs at least 3 vertices and 1 triangle";
  fe.nv = mesh->nv;
  fe.nt = mesh->nt;
  const int nv = fe.nv, nt = fe.nt;
  fe.xy.assign(mesh->xy, mesh->xy + 2 * (size_t)nv);
  fe.tri.assign(mesh->tri, mesh->tri + 3 * (size_t)nt);
  for (int t = 0; t < 3 * nt; ++t)
    if (fe.tri[t] < 0 || fe.tri[t] >= nv) return "triangle vertex index out of range";

  // geometry: gradients of the barycentric coordinates and twice the area
  fe.geom.assign((size_t)nt * 8, 0.0);
  for (int e = 0; e < nt; ++e) {
    const int* v = &fe.tri[3 * e];
    double x0 = fe.xy[2 * v[0]], y0 = fe.xy[2 * v[0] + 1];
    double x1 = fe.xy[2 * v[1]], y1 = fe.xy[2 * v[1] + 1];
    double x2 = fe.xy[2 * v[2]], y2 = fe.xy[2 * v[2] + 1];
    double det = (x1 - x0) * (y2 - y0) - (x2 - x0) * (y1 - y0);
    if (!(det > 0.0)) return "triangle " + std::to_string(e) + " is not counter-clockwise";
    double* g = &fe.geom[8 * (size_t)e];
    g[0] = (y1 - y2) / det; g[1] = (x2 - x1) / det;
    g[2] = (y2 - y0) / det; g[3] = (x0 - x2) / det;
    g[4] = (y0 - y1) / det; g[5] = (x1 - x0) / det;
    g[6] = det;
  }

  // edges and P2 numbering
  std::vector<long long> ekeys((size_t)nt * 3);
  for (int e = 0; e < nt; ++e)
    for (int l = 0; l < 3; ++l) {
      long long a = fe.tri[3 * e + LE[l][0]], b = fe.tri[3 * e + LE[l][1]];
      if (a == b) return "degenerate triangle";
      if (a > b) std::swap(a, b);
      ekeys[3 * (size_t)e + l] = a * nv + b;
    }
  std::vector<int> eid;
  unique_keys(ekeys, fe.edges, eid);
  fe.ne = (int)fe.edges.size();
  fe.n2 = nv + fe.ne;
  fe.np = element == 1 ? 3 * nt : nv;
  // pressure dof of local vertex i on triangle e
  auto prow = [&](int e, int i) -> long long {
    return element == 1 ? 3LL * e + i : (long long)fe.tri[3 * e + i];
  };
  fe.edge_count.assign(fe.ne, 0);
  for (int id : eid) fe.edge_count[id]++;
  for (int c : fe.edge_count)
    if (c > 2) return "non-manifold edge (shared by more than two triangles)";
  fe.dofs.resize((size_t)nt * 6);
  for (int e = 0; e < nt; ++e) {
    for (int l = 0; l < 3; ++l) fe.dofs[6 * (size_t)e + l] = fe.tri[3 * e + l];
    for (int l = 0; l < 3; ++l) fe.dofs[6 * (size_t)e + 3 + l] = nv + eid[3 * (size_t)e + l];
  }
  fe.node_xy.resize(2 * (size_t)fe.n2);
  std::copy(fe.xy.begin(), fe.xy.end(), fe.node_xy.begin());
  fe.is_bnd.assign(fe.n2, 0);
  for (int k = 0; k < fe.ne; ++k) {
    long long a = fe.edges[k] / nv, b = fe.edges[k] % nv;
    fe.node_xy[2 * (size_t)(nv + k)] = 0.5 * (fe.xy[2 * a] + fe.xy[2 * b]);
    fe.node_xy[2 * (size_t)(nv + k) + 1] = 0.5 * (fe.xy[2 * a + 1] + fe.xy[2 * b + 1]);
    if (fe.edge_count[k] == 1) {
      fe.is_bnd[a] = fe.is_bnd[b] = fe.is_bnd[nv + k] = 1;
    }
  }
  fe.bnd_nodes.clear();
  for (int k = 0; k < fe.n2; ++k)
    if (fe.is_bnd[k]) fe.bnd_nodes.push_back(k);

  // F pattern and scatter map
  {
    std::vector<long long> keys((size_t)nt * 36);
    for (int e = 0; e < nt; ++e)
      for (int a = 0; a < 6; ++a)
        for (int b = 0; b < 6; ++b)
          keys[36 * (size_t)e + 6 * a + b] =
              (long long)fe.dofs[6 * (size_t)e + a] * fe.n2 + fe.dofs[6 * (size_t)e + b];
    std::vector<long long> uniq;
    unique_keys(keys, uniq, fe.f_slot_nnz);
    csr_from_keys(uniq, fe.n2, fe.n2, fe.F);
    invert_map(fe.f_slot_nnz, fe.F.nnz(), fe.f_gather_ptr, fe.f_gather_slot);
    fe.f_diag.assign(fe.n2, -1);
    for (int r = 0; r < fe.n2; ++r)
      for (int k = fe.F.rowptr[r]; k < fe.F.rowptr[r + 1]; ++k)
        if (fe.F.col[k] == r) fe.f_diag[r] = k;
  }
  // B pattern (P1 rows x P2 columns) and scatter map
  {
    std::vector<long long> keys((size_t)nt * 18);
    for (int e = 0; e < nt; ++e)
      for (int i = 0; i < 3; ++i)
        for (int a = 0; a < 6; ++a)
          keys[18 * (size_t)e + 6 * i + a] = prow(e, i) * fe.n2 + fe.dofs[6 * (size_t)e + a];
    std::vector<long long> uniq;
    std::vector<int> slot_nnz;
    unique_keys(keys, uniq, slot_nnz);
    csr_from_keys(uniq, fe.np, fe.n2, fe.B);
    invert_map(slot_nnz, fe.B.nnz(), fe.b_gather_ptr, fe.b_gather_slot);
    // transpose pattern
    std::vector<long long> tkeys(uniq.size());
    for (size_t k = 0; k < uniq.size(); ++k) {
      long long i = uniq[k] / fe.n2, a = uniq[k] % fe.n2;
      tkeys[k] = a * fe.np + i;
    }
    std::vector<long long> tuniq;
    std::vector<int> where;
    unique_keys(tkeys, tuniq, where);
    csr_from_keys(tuniq, fe.n2, fe.np, fe.BT);
    fe.bt_src.assign(uniq.size(), 0);
    for (size_t k = 0; k < uniq.size(); ++k) fe.bt_src[where[k]] = (int)k;
  }
  // node -> element-local slots
  {
    std::vector<int> slot_node((size_t)nt * 6);
    for (size_t s = 0; s < slot_node.size(); ++s) slot_node[s] = fe.dofs[s];
    invert_map(slot_node, fe.n2, fe.node_ptr, fe.node_slot);
  }
  // lumped pressure mass: area / 3 per local vertex, summed per pressure dof
  fe.mp_lumped.assign(fe.np, 0.0);
  for (int e = 0; e < nt; ++e)
    for (int i = 0; i < 3; ++i) fe.mp_lumped[prow(e, i)] += 0.5 * fe.geom[8 * (size_t)e + 6] / 3.0;
  // pressure Laplacian of the continuous pressure (P1 stiffness, node 0 pinned)
  if (element == 0) {
    std::vector<long long> keys((size_t)nt * 9);
    std::vector<double> vals((size_t)nt * 9);
    for (int e = 0; e < nt; ++e) {
      const double* g = &fe.geom[8 * (size_t)e];
      double area = 0.5 * g[6];
      for (int i = 0; i < 3; ++i) {
        for (int k = 0; k < 3; ++k) {
          keys[9 * (size_t)e + 3 * i + k] = (long long)fe.tri[3 * e + i] * fe.np + fe.tri[3 * e + k];
          vals[9 * (size_t)e + 3 * i + k] = area * (g[2 * i] * g[2 * k] + g[2 * i + 1] * g[2 * k + 1]);
        }
      }
    }
    std::vector<long long> uniq;
    std::vector<int> where;
    unique_keys(keys, uniq, where);
    csr_from_keys(uniq, fe.np, fe.np, fe.Kp);
    fe.Kp.val.assign(uniq.size(), 0.0);
    // deterministic: slots in ascending order per nnz
    invert_map(where, (long long)uniq.size(), fe.p1_gather_ptr, fe.p1_gather_slot);
    const std::vector<int>& ptr = fe.p1_gather_ptr;
    const std::vector<int>& slots = fe.p1_gather_slot;
    for (size_t k = 0; k < uniq.size(); ++k)
      for (int t = ptr[k]; t < ptr[k + 1]; ++t) fe.Kp.val[k] += vals[slots[t]];
    // pin node 0: identity row and column
    for (int r = 0; r < fe.np; ++r)
      for (int k = fe.Kp.rowptr[r]; k < fe.Kp.rowptr[r + 1]; ++k) {
        int c = fe.Kp.col[k];
        if (r == 0 || c == 0) fe.Kp.val[k] = (r == c) ? 1.0 : 0.0;
      }
  }
  return "";
}

// ------------------------------------------------------------------------- AMG
namespace {

void csr_transpose(const HostCsr& A, HostCsr& T) {
  T.nrows = A.ncols;
  T.ncols = A.nrows;
  T.rowptr.assign(T.nrows + 1, 0);
  for (int c : A.col) T.rowptr[c + 1]++;
  for (int r = 0; r < T.nrows; ++r) T.rowptr[r + 1] += T.rowptr[r];
  std::vector<int> fill(T.rowptr.begin(), T.rowptr.end() - 1);
  T.col.resize(A.col.size());
  T.val.resize(A.col.size());
  for (int r = 0; r < A.nrows; ++r)
    for (int k = A.rowptr[r]; k < A.rowptr[r + 1]; ++k) {
      int p = fill[A.col[k]]++;
      T.col[p] = r;
      T.val[p] = A.val[k];
    }
}

// C = A B (Gustavson, columns sorted per row)
void csr_matmul(const HostCsr& A, const HostCsr& B, HostCsr& C) {
  C.nrows = A.nrows;
  C.ncols = B.ncols;
  C.rowptr.assign(C.nrows + 1, 0);
  C.col.clear();
  C.val.clear();
  std::vector<int> mark(B.ncols, -1);
  std::vector<double> acc(B.ncols, 0.0);
  std::vector<int> cols;
  for (int r = 0; r < A.nrows; ++r) {
    cols.clear();
    for (int k = A.rowptr[r]; k < A.rowptr[r + 1]; ++k) {
      int a = A.col[k];
      double av = A.val[k];
      for (int t = B.rowptr[a]; t < B.rowptr[a + 1]; ++t) {
        int c = B.col[t];
        if (mark[c] != r) {
          mark[c] = r;
          acc[c] = 0.0;
          cols.push_back(c);
        }
        acc[c] += av * B.val[t];
      }
    }
    std::sort(cols.begin(), cols.end());
    for (int c : cols) {
      C.col.push_back(c);
      C.val.push_back(acc[c]);
    }
    C.rowptr[r + 1] = (int)C.col.size();
  }
}

double spectral_radius_DinvA(const HostCsr& A, const std::vector<double>& dinv) {
  int n = A.nrows;
  std::vector<double> x(n), y(n);
  for (int i = 0; i < n; ++i) x[i] = 1.0 + 0.37 * std::sin(1.7 * i + 0.3);
  double lam = 1.0;
  for (int it = 0; it < 30; ++it) {
    double nx = 0.0;
    for (int i = 0; i < n; ++i) nx += x[i] * x[i];
    nx = std::sqrt(nx);
    for (int i = 0; i < n; ++i) x[i] /= nx;
    for (int i = 0; i < n; ++i) {
      double s = 0.0;
      for (int k = A.rowptr[i]; k < A.rowptr[i + 1]; ++k) s += A.val[k] * x[A.col[k]];
      y[i] = dinv[i] * s;
    }
    double ny = 0.0;
    for (int i = 0; i < n; ++i) ny += y[i] * y[i];
    lam = std::sqrt(ny);
    x.swap(y);
  }
  return lam * 1.05;
}

std::vector<double> diag_inv(const HostCsr& A) {
  std::vector<double> d(A.nrows, 0.0);
  for (int r = 0; r < A.nrows; ++r)
    for (int k = A.rowptr[r]; k < A.rowptr[r + 1]; ++k)
      if (A.col[k] == r) d[r] = A.val[k];
  for (auto& v : d) v = (v != 0.0) ? 1.0 / v : 0.0;
  return d;
}

// Greedy aggregation on the strength graph |a_ij| >= theta sqrt(|a_ii a_jj|).
int aggregate(const HostCsr& A, double theta, std::vector<int>& agg) {
  int n = A.nrows;
  std::vector<double> diag(n, 0.0);
  for (int r = 0; r < n; ++r)
    for (int k = A.rowptr[r]; k < A.rowptr[r + 1]; ++k)
      if (A.col[k] == r) diag[r] = std::fabs(A.val[k]);
  std::vector<std::vector<int>> S(n);
  for (int r = 0; r < n; ++r)
    for (int k = A.rowptr[r]; k < A.rowptr[r + 1]; ++k) {
      int c = A.col[k];
      if (c != r && std::fabs(A.val[k]) >= theta * std::sqrt(diag[r] * diag[c]) && A.val[k] != 0.0)
        S[r].push_back(c);
    }
  agg.assign(n, -1);
  int na = 0;
  for (int i = 0; i < n; ++i) {         // pass 1: whole free neighbourhoods
    if (agg[i] >= 0) continue;
    bool free_nb = true;
    for (int c : S[i])
      if (agg[c] >= 0) { free_nb = false; break; }
    if (!free_nb) continue;
    agg[i] = na;
    for (int c : S[i]) agg[c] = na;
    na++;
  }
  std::vector<int> agg1 = agg;
  for (int i = 0; i < n; ++i) {         // pass 2: join a neighbouring aggregate
    if (agg[i] >= 0) continue;
    for (int c : S[i])
      if (agg1[c] >= 0) { agg[i] = agg1[c]; break; }
  }
  for (int i = 0; i < n; ++i) {         // pass 3: leftovers
    if (agg[i] >= 0) continue;
    agg[i] = na;
    for (int c : S[i])
      if (agg[c] < 0) agg[c] = na;
    na++;
  }
  return na;
}

bool dense_inverse(int n, std::vector<double> A, std::vector<double>& inv) {
  inv.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) inv[(size_t)i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[(size_t)r * n + c]) > std::fabs(A[(size_t)p * n + c])) p = r;
    if (A[(size_t)p * n + c] == 0.0) return false;
    if (p != c)
      for (int k = 0; k < n; ++k) {
        std::swap(A[(size_t)p * n + k], A[(size_t)c * n + k]);
        std::swap(inv[(size_t)p * n + k], inv[(size_t)c * n + k]);
      }
    double d = 1.0 / A[(size_t)c * n + c];
    for (int k = 0; k < n; ++k) {
      A[(size_t)c * n + k] *= d;
      inv[(size_t)c * n + k] *= d;
    }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      double f = A[(size_t)r * n + c];
      if (f == 0.0) continue;
      for (int k = 0; k < n; ++k) {
        A[(size_t)r * n + k] -= f * A[(size_t)c * n + k];
        inv[(size_t)r * n + k] -= f * inv[(size_t)c * n + k];
      }
    }
  }
  return true;
}

}  // namespace

std::string build_algebraic_laplacian(FeHost& fe) {
  const int nt = fe.nt, n2 = fe.n2, np = fe.np;
  // D: the diagonal of the P2 mass matrix scaled on every triangle so that
  // its entries sum to the area (vertices area/19, edge midpoints
  // 16 area/57: the diagonal entries area/30 and 8 area/45 times 30/19)
  std::vector<double> D(n2, 0.0);
  for (int e = 0; e < nt; ++e) {
    const double area = 0.5 * fe.geom[8 * (size_t)e + 6];
    for (int a = 0; a < 3; ++a) D[fe.dofs[6 * (size_t)e + a]] += area / 19.0;
    for (int a = 3; a < 6; ++a) D[fe.dofs[6 * (size_t)e + a]] += 16.0 * area / 57.0;
  }
  fe.lsc_dinv.assign(n2, 0.0);
  for (int k = 0; k < n2; ++k)
    if (!fe.is_bnd[k] && D[k] > 0.0) fe.lsc_dinv[k] = 1.0 / D[k];
  // element values of B_d (slot 18e + 6i + a): -(d phi_a / d x_d, lambda_i),
  // integrated exactly with (lambda_i, lambda_k) = area (1 + delta_ik) / 12:
  // vertex a: -(area/3) delta_ai grad lambda_a; midpoint of edge (p, q):
  // -(area/3) ((1 + delta_pi) grad lambda_q + (1 + delta_qi) grad lambda_p)
  std::vector<double> loc[2] = {std::vector<double>((size_t)nt * 18), std::vector<double>((size_t)nt * 18)};
  for (int e = 0; e < nt; ++e) {
    const double* g = &fe.geom[8 * (size_t)e];
    const double a3 = 0.5 * g[6] / 3.0;
    for (int i = 0; i < 3; ++i)
      for (int d = 0; d < 2; ++d) {
        double* v = &loc[d][18 * (size_t)e + 6 * i];
        for (int a = 0; a < 3; ++a) v[a] = (a == i) ? -a3 * g[2 * a + d] : 0.0;
        for (int l = 0; l < 3; ++l) {
          const int p = LE[l][0], q = LE[l][1];
          v[3 + l] = -a3 * ((1.0 + (p == i)) * g[2 * q + d] + (1.0 + (q == i)) * g[2 * p + d]);
        }
      }
  }
  // Bs = [Bx | By] (np x 2 n2), assembled in B's pattern (slots summed in
  // ascending order), and W = diag(D^{-1}, D^{-1}) Bs^T
  const long long nb = fe.B.nnz();
  HostCsr Bs;
  Bs.nrows = np;
  Bs.ncols = 2 * n2;
  Bs.rowptr.assign(np + 1, 0);
  Bs.col.resize(2 * (size_t)nb);
  Bs.val.resize(2 * (size_t)nb);
  for (int r = 0; r < np; ++r) {
    const int k0 = fe.B.rowptr[r], k1 = fe.B.rowptr[r + 1];
    const size_t o = 2 * (size_t)k0;
    for (int d = 0; d < 2; ++d)
      for (int k = k0; k < k1; ++k) {
        double sum = 0.0;
        for (int t = fe.b_gather_ptr[k]; t < fe.b_gather_ptr[k + 1]; ++t) sum += loc[d][fe.b_gather_slot[t]];
        const size_t w = o + (size_t)d * (k1 - k0) + (k - k0);
        Bs.col[w] = fe.B.col[k] + d * n2;
        Bs.val[w] = sum;
      }
    Bs.rowptr[r + 1] = 2 * k1;
  }
  HostCsr W;
  csr_transpose(Bs, W);
  for (int r = 0; r < W.nrows; ++r)
    for (int k = W.rowptr[r]; k < W.rowptr[r + 1]; ++k) W.val[k] *= fe.lsc_dinv[r % n2];
  csr_matmul(Bs, W, fe.Kp);
  // pin dof 0: identity row and column
  for (int r = 0; r < np; ++r)
    for (int k = fe.Kp.rowptr[r]; k < fe.Kp.rowptr[r + 1]; ++k) {
      const int c = fe.Kp.col[k];
      if (r == 0 || c == 0) fe.Kp.val[k] = (r == c) ? 1.0 : 0.0;
    }
  for (int r = 1; r < np; ++r) {
    bool diag = false;
    for (int k = fe.Kp.rowptr[r]; k < fe.Kp.rowptr[r + 1]; ++k)
      if (fe.Kp.col[k] == r && fe.Kp.val[k] > 0.0) diag = true;
    if (!diag) return "pressure dof " + std::to_string(r) + " is not coupled to any interior velocity node";
  }
  fe.p1_gather_ptr.clear();
  fe.p1_gather_slot.clear();
  return "";
}

namespace {

// Smoother blocks of the discontinuous pressure: the nine dofs of every macro
// triangle when the mesh is a barycenter refinement (every triangle has one
// vertex that is interior, has exactly three triangles around it and sits at
// the mean of their other vertices), else the three dofs of every triangle.
void pressure_blocks(const FeHost& fe, int& bs, std::vector<int>& idx, std::vector<int>* macro_out = nullptr) {
  const int nv = fe.nv, nt = fe.nt;
  std::vector<int> cnt(nv + 1, 0);
  for (int t = 0; t < 3 * nt; ++t) cnt[fe.tri[t] + 1]++;
  for (int v = 0; v < nv; ++v) cnt[v + 1] += cnt[v];
  std::vector<int> fill(cnt.begin(), cnt.end() - 1), vt(3 * (size_t)nt);
  for (int t = 0; t < 3 * nt; ++t) vt[fill[fe.tri[t]]++] = t / 3;
  std::vector<int> owner(nt, -1);
  std::vector<int> macro;
  bool ok = true;
  for (int v = 0; v < nv && ok; ++v) {
    if (fe.is_bnd[v] || cnt[v + 1] - cnt[v] != 3) continue;
    int ts[3] = {vt[cnt[v]], vt[cnt[v] + 1], vt[cnt[v] + 2]};
    double mx = 0.0, my = 0.0, ext = 0.0;
    for (int k = 0; k < 3; ++k)
      for (int l = 0; l < 3; ++l) {
        int u = fe.tri[3 * ts[k] + l];
        if (u == v) continue;
        mx += fe.xy[2 * u] / 6.0;          // each outer vertex is seen from two triangles
        my += fe.xy[2 * u + 1] / 6.0;
        ext = std::max(ext, std::fabs(fe.xy[2 * u] - fe.xy[2 * v]) + std::fabs(fe.xy[2 * u + 1] - fe.xy[2 * v + 1]));
      }
    if (std::fabs(mx - fe.xy[2 * v]) + std::fabs(my - fe.xy[2 * v + 1]) > 1e-9 * ext) continue;
    for (int k = 0; k < 3; ++k) {
      if (owner[ts[k]] >= 0) ok = false;
      owner[ts[k]] = v;
      macro.push_back(ts[k]);
    }
  }
  for (int t = 0; t < nt && ok; ++t)
    if (owner[t] < 0) ok = false;
  idx.clear();
  if (macro_out) *macro_out = ok ? macro : std::vector<int>();
  if (ok) {
    bs = 9;
    for (int t : macro)
      for (int i = 0; i < 3; ++i) idx.push_back(3 * t + i);
  } else {
    bs = 3;
    for (int d = 0; d < 3 * nt; ++d) idx.push_back(d);
  }
}

double spectral_radius_BinvA(const HostCsr& A, int bs, const std::vector<int>& idx, const std::vector<double>& inv) {
  const int n = A.nrows, nb = n / bs;
  std::vector<double> x(n), y(n), ax(n);
  for (int i = 0; i < n; ++i) x[i] = 1.0 + 0.37 * std::sin(1.7 * i + 0.3);
  double lam = 1.0;
  for (int it = 0; it < 40; ++it) {
    double nx = 0.0;
    for (double v : x) nx += v * v;
    nx = std::sqrt(nx);
    for (double& v : x) v /= nx;
    for (int i = 0; i < n; ++i) {
      double s = 0.0;
      for (int k = A.rowptr[i]; k < A.rowptr[i + 1]; ++k) s += A.val[k] * x[A.col[k]];
      ax[i] = s;
    }
    for (int b = 0; b < nb; ++b)
      for (int i = 0; i < bs; ++i) {
        double s = 0.0;
        for (int j = 0; j < bs; ++j) s += inv[((size_t)b * bs + i) * bs + j] * ax[idx[(size_t)b * bs + j]];
        y[idx[(size_t)b * bs + i]] = s;
      }
    double ny = 0.0;
    for (double v : y) ny += v * v;
    lam = std::sqrt(ny);
    x.swap(y);
  }
  return lam * 1.05;
}

}  // namespace

std::string build_amg(FeHost& fe, int coarse_max) {
  AmgHost& amg = fe.amg;
  amg.levels.clear();
  AmgLevelHost L0;
  L0.A = fe.Kp;
  amg.levels.push_back(L0);
  for (int lev = 0; lev < 25; ++lev) {
    AmgLevelHost& L = amg.levels.back();
    L.dinv = diag_inv(L.A);
    int n = L.A.nrows;
    // the finest level of the discontinuous pressure is smoothed by blocks
    // (below), so its point-Jacobi damping is never used and not estimated
    const bool blocks = lev == 0 && fe.element == 1 && n > coarse_max;
    L.omega = blocks ? 0.0 : 4.0 / (3.0 * spectral_radius_DinvA(L.A, L.dinv));
    if (n <= coarse_max) break;
    if (lev == 0 && fe.element == 0) {
      // continuous pressure on a barycenter refinement: the first coarse space
      // is P1 on the parent mesh (a parent vertex keeps its value, a
      // barycenter takes the mean of its triangle's three vertices; the
      // pinned node 0 takes none), then smoothed aggregation as usual
      int bs = 0;
      std::vector<int> idx, macro;
      pressure_blocks(fe, bs, idx, &macro);
      if (bs == 9) {
        std::vector<char> is_bary(fe.nv, 0);
        std::vector<int> outer((size_t)fe.nv * 3, -1);
        for (size_t q = 0; q < macro.size(); q += 3) {
          const int t0 = macro[q];
          int g = -1;
          for (int l = 0; l < 3 && g < 0; ++l) {       // the vertex shared by the three children
            const int v = fe.tri[3 * t0 + l];
            bool all = true;
            for (int k = 1; k < 3; ++k) {
              const int t = macro[q + k];
              all = all && (fe.tri[3 * t] == v || fe.tri[3 * t + 1] == v || fe.tri[3 * t + 2] == v);
            }
            if (all) g = v;
          }
          is_bary[g] = 1;
          int no = 0;
          for (int k = 0; k < 3; ++k)
            for (int l = 0; l < 3; ++l) {
              const int u = fe.tri[3 * macro[q + k] + l];
              bool seen = (u == g);
              for (int o = 0; o < no; ++o) seen = seen || outer[(size_t)g * 3 + o] == u;
              if (!seen && no < 3) outer[(size_t)g * 3 + no++] = u;
            }
        }
        std::vector<int> coarse(fe.nv, -1);
        int nc = 0;
        for (int v = 0; v < fe.nv; ++v)
          if (!is_bary[v]) coarse[v] = nc++;
        HostCsr P;
        P.nrows = n;
        P.ncols = nc;
        P.rowptr.assign(n + 1, 0);
        for (int v = 0; v < n; ++v) {
          if (v != 0) {
            if (!is_bary[v]) {
              P.col.push_back(coarse[v]);
              P.val.push_back(1.0);
            } else {
              int cs[3] = {coarse[outer[(size_t)v * 3]], coarse[outer[(size_t)v * 3 + 1]],
                           coarse[outer[(size_t)v * 3 + 2]]};
              std::sort(cs, cs + 3);
              for (int k = 0; k < 3; ++k) {
                P.col.push_back(cs[k]);
                P.val.push_back(1.0 / 3.0);
              }
            }
          }
          P.rowptr[v + 1] = (int)P.col.size();
        }
        HostCsr R, RA, Ac;
        csr_transpose(P, R);
        csr_matmul(R, L.A, RA);
        csr_matmul(RA, P, Ac);
        L.P = P;
        L.R = R;
        AmgLevelHost next;
        next.A = Ac;
        amg.levels.push_back(next);
        continue;
      }
    }
    if (lev == 0 && fe.element == 1) {
      // discontinuous pressure: the first coarse space is the continuous P1
      // space on the mesh vertices, injected into P1disc (P: dof 3t + i takes
      // the value at vertex tri[3t + i]; the pinned dof 0 takes none), and
      // the fine level is smoothed by block Jacobi over macro triangles
      HostCsr P;
      P.nrows = n;
      P.ncols = fe.nv;
      P.rowptr.assign(n + 1, 0);
      for (int d = 0; d < n; ++d) {
        if (d != 0) {
          P.col.push_back(fe.tri[d]);
          P.val.push_back(1.0);
        }
        P.rowptr[d + 1] = (int)P.col.size();
      }
      pressure_blocks(fe, L.bs, L.blk_idx);
      const int bs = L.bs, nb = n / bs;
      std::vector<int> pos(n, -1);
      L.blk_inv.assign((size_t)nb * bs * bs, 0.0);
      for (int b = 0; b < nb; ++b) {
        for (int i = 0; i < bs; ++i) pos[L.blk_idx[(size_t)b * bs + i]] = i;
        std::vector<double> blk((size_t)bs * bs, 0.0), inv;
        for (int i = 0; i < bs; ++i) {
          const int r = L.blk_idx[(size_t)b * bs + i];
          for (int k = L.A.rowptr[r]; k < L.A.rowptr[r + 1]; ++k)
            if (pos[L.A.col[k]] >= 0) blk[(size_t)i * bs + pos[L.A.col[k]]] = L.A.val[k];
        }
        for (int i = 0; i < bs; ++i) pos[L.blk_idx[(size_t)b * bs + i]] = -1;
        if (!dense_inverse(bs, blk, inv)) return "singular pressure smoother block " + std::to_string(b);
        std::copy(inv.begin(), inv.end(), L.blk_inv.begin() + (size_t)b * bs * bs);
      }
      L.blk_omega = 1.6 / spectral_radius_BinvA(L.A, bs, L.blk_idx, L.blk_inv);
      HostCsr R, RA, Ac;
      csr_transpose(P, R);
      csr_matmul(R, L.A, RA);
      csr_matmul(RA, P, Ac);
      L.P = P;
      L.R = R;
      AmgLevelHost next;
      next.A = Ac;
      amg.levels.push_back(next);
      continue;
    }
    std::vector<int> agg;
    int na = aggregate(L.A, 0.08, agg);
    if (na >= n || na < 1) break;
    // tentative prolongator: normalized piecewise constants
    std::vector<int> size(na, 0);
    for (int a : agg) size[a]++;
    HostCsr Pt;
    Pt.nrows = n;
    Pt.ncols = na;
    Pt.rowptr.resize(n + 1);
    Pt.col.resize(n);
    Pt.val.resize(n);
    for (int i = 0; i < n; ++i) {
      Pt.rowptr[i] = i;
      Pt.col[i] = agg[i];
      Pt.val[i] = 1.0 / std::sqrt((double)size[agg[i]]);
    }
    Pt.rowptr[n] = n;
    // smoothed prolongator P = (I - omega D^-1 A) Pt
    HostCsr AP;
    csr_matmul(L.A, Pt, AP);
    HostCsr P;
    P.nrows = n;
    P.ncols = na;
    P.rowptr.assign(n + 1, 0);
    for (int i = 0; i < n; ++i) {
      std::vector<std::pair<int, double>> row;
      for (int k = AP.rowptr[i]; k < AP.rowptr[i + 1]; ++k)
        row.push_back({AP.col[k], -L.omega * L.dinv[i] * AP.val[k]});
      row.push_back({agg[i], Pt.val[i]});
      std::sort(row.begin(), row.end());
      int last = -1;
      for (auto& pr : row) {
        if (pr.first == last) {
          P.val.back() += pr.second;
        } else {
          P.col.push_back(pr.first);
          P.val.push_back(pr.second);
          last = pr.first;
        }
      }
      P.rowptr[i + 1] = (int)P.col.size();
    }
    HostCsr R, RA, Ac;
    csr_transpose(P, R);
    csr_matmul(R, L.A, RA);
    csr_matmul(RA, P, Ac);
    L.P = P;
    L.R = R;
    AmgLevelHost next;
    next.A = Ac;
    amg.levels.push_back(next);
  }
  AmgLevelHost& C = amg.levels.back();
  amg.nc = C.A.nrows;
  if (C.dinv.empty()) {
    C.dinv = diag_inv(C.A);
    C.omega = 4.0 / (3.0 * spectral_radius_DinvA(C.A, C.dinv));
  }
  if (amg.nc > 4096) return "pressure-Laplacian hierarchy did not coarsen below 4096 unknowns";
  std::vector<double> dense((size_t)amg.nc * amg.nc, 0.0);
  for (int r = 0; r < amg.nc; ++r)
    for (int k = C.A.rowptr[r]; k < C.A.rowptr[r + 1]; ++k)
      dense[(size_t)r * amg.nc + C.A.col[k]] = C.A.val[k];
  if (!dense_inverse(amg.nc, dense, amg.coarse_inv)) return "coarsest pressure operator is singular";
  return "";
}

// ------------------------------------------------------------- small dense
void eig_sym(int n, const double* A0, double* w, double* U) {
  // cyclic Jacobi rotations
  std::vector<double> A(A0, A0 + (size_t)n * n);
  for (int i = 0; i < n * n; ++i) U[i] = 0.0;
  for (int i = 0; i < n; ++i) U[i * n + i] = 1.0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        double a = A[i * n + j] * A[i * n + j];
        tot += a;
        if (i != j) off += a;
      }
    if (off <= 1e-30 * tot || off == 0.0) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        double apq = A[p * n + q];
        if (apq == 0.0) continue;
        double app = A[p * n + p], aqq = A[q * n + q];
        double theta = 0.5 * (aqq - app) / apq;
        double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {
          double akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = c * akp - s * akq;
          A[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {
          double apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = c * apk - s * aqk;
          A[q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          double ukp = U[k * n + p], ukq = U[k * n + q];
          U[k * n + p] = c * ukp - s * ukq;
          U[k * n + q] = s * ukp + c * ukq;
        }
      }
  }
  // sort descending
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::vector<double> d(n);
  for (int i = 0; i < n; ++i) d[i] = A[i * n + i];
  std::sort(order.begin(), order.end(), [&](int a, int b) { return d[a] > d[b]; });
  std::vector<double> U2((size_t)n * n);
  for (int j = 0; j < n; ++j) {
    w[j] = d[order[j]];
    for (int i = 0; i < n; ++i) U2[i * n + j] = U[i * n + order[j]];
  }
  std::copy(U2.begin(), U2.end(), U);
}

// Cholesky QR factors of a full-rank r-column Gram matrix G = R^T R:
// T_ = R^{-1}, S_ = R (the same conventions as svqb: W T_ has orthonormal
// columns, W = (W T_) S_).  Used only when full rank is certain: lambda_max
// <= trace(G) and lambda_min >= 1 / ||R^{-1}||_F^2, so trace(G) ||R^{-1}||_F^2
// < 1e-2 / thresh means every eigenvalue is above 100 thresh lambda_max and
// svqb would keep all r directions.  About a hundred times cheaper than the
// eigen-decomposition, which sits on the critical path of every block
// iteration.  Returns false (and leaves T_, S_ unspecified) otherwise.
bool cholqr_factors(int r, const std::vector<double>& G, double thresh, std::vector<double>& Tm,
                           std::vector<double>& Sm) {
  std::vector<double> R((size_t)r * r, 0.0);          // upper triangular, G = R^T R
  double tr = 0.0;
  for (int i = 0; i < r; ++i) tr += G[(size_t)i * r + i];
  if (!(tr > 0.0)) return false;
  for (int j = 0; j < r; ++j) {
    double d = G[(size_t)j * r + j];
    for (int k = 0; k < j; ++k) d -= R[(size_t)k * r + j] * R[(size_t)k * r + j];
    if (!(d > 0.0)) return false;
    const double rjj = std::sqrt(d);
    R[(size_t)j * r + j] = rjj;
    for (int i = j + 1; i < r; ++i) {
      double v = G[(size_t)j * r + i];
      for (int k = 0; k < j; ++k) v -= R[(size_t)k * r + j] * R[(size_t)k * r + i];
      R[(size_t)j * r + i] = v / rjj;
    }
  }
  // R^{-1} (upper triangular), column by column by back substitution
  std::vector<double> Ri((size_t)r * r, 0.0);
  double fro = 0.0;
  for (int c = 0; c < r; ++c) {
    for (int i = c; i >= 0; --i) {
      double v = (i == c) ? 1.0 : 0.0;
      for (int k = i + 1; k <= c; ++k) v -= R[(size_t)i * r + k] * Ri[(size_t)k * r + c];
      v /= R[(size_t)i * r + i];
      Ri[(size_t)i * r + c] = v;
      fro += v * v;
    }
  }
  if (!(tr * fro < 1e-2 / thresh)) return false;
  Tm.swap(Ri);
  Sm.swap(R);
  return true;
}

void BlockLS::init(int r_, int J_, int m_, const double* S0) {
  r = r_;
  J = J_;
  m = m_;
  k = 0;
  ldr = m * r;
  // every entry of R and hv that is read is written first
  R.resize((size_t)ldr * ldr);
  hv.resize((size_t)m * r * 2 * r);
  htau.assign((size_t)m * r, 0.0);
  g.assign((size_t)(m + 1) * r * J, 0.0);
  for (int i = 0; i < r; ++i)
    for (int j = 0; j < J; ++j) g[(size_t)i * J + j] = S0[(size_t)i * J + j];
  c.resize((size_t)(m + 1) * r * r);
  s.resize((size_t)std::max(r, J));
}

// Householder QR of the block Hessenberg matrix, one block column at a time:
// the previous reflectors are applied to the new column, then r new ones
// (each spanning 2r rows) annihilate its subdiagonal block and are applied to
// the right-hand sides.  Every inner loop runs over the r columns of the
// block (or the J right-hand sides), contiguous in memory.
bool BlockLS::add(const double* h) {
  const int rows = (k + 2) * r;
  std::copy(h, h + (size_t)rows * r, c.begin());
  double* sv = s.data();
  for (int col = 0; col < k * r; ++col) {
    const double tau = htau[col];
    if (tau == 0.0) continue;
    const int lo = col, len = (col / r + 2) * r - col;
    const double* v = &hv[(size_t)col * 2 * r];
    for (int t = 0; t < r; ++t) sv[t] = 0.0;
    for (int i = 0; i < len; ++i) {
      const double a = v[i];
      const double* row = &c[(size_t)(lo + i) * r];
      for (int t = 0; t < r; ++t) sv[t] += a * row[t];
    }
    for (int t = 0; t < r; ++t) sv[t] *= tau;
    for (int i = 0; i < len; ++i) {
      const double a = v[i];
      double* row = &c[(size_t)(lo + i) * r];
      for (int t = 0; t < r; ++t) row[t] -= a * sv[t];
    }
  }
  bool ok = true;
  for (int t = 0; t < r; ++t) {
    const int col = k * r + t;
    const int lo = col, hi = (k + 2) * r, len = hi - lo;
    double* v = &hv[(size_t)col * 2 * r];
    for (int i = 0; i < 2 * r; ++i) v[i] = 0.0;
    const double alpha = c[(size_t)lo * r + t];
    double nrm2 = 0.0;
    for (int i = lo; i < hi; ++i) nrm2 += c[(size_t)i * r + t] * c[(size_t)i * r + t];
    const double nrm = std::sqrt(nrm2);
    if (nrm == 0.0) {
      htau[col] = 0.0;
      ok = false;
      continue;
    }
    const double beta = (alpha >= 0) ? -nrm : nrm;
    const double denom = alpha - beta;
    v[0] = 1.0;
    for (int i = lo + 1; i < hi; ++i) v[i - lo] = c[(size_t)i * r + t] / denom;
    const double tau = (beta - alpha) / beta;
    htau[col] = tau;
    c[(size_t)lo * r + t] = beta;
    for (int i = lo + 1; i < hi; ++i) c[(size_t)i * r + t] = 0.0;
    // the remaining columns of this block
    if (t + 1 < r) {
      for (int t2 = t + 1; t2 < r; ++t2) sv[t2] = 0.0;
      for (int i = 0; i < len; ++i) {
        const double a = v[i];
        const double* row = &c[(size_t)(lo + i) * r];
        for (int t2 = t + 1; t2 < r; ++t2) sv[t2] += a * row[t2];
      }
      for (int t2 = t + 1; t2 < r; ++t2) sv[t2] *= tau;
      for (int i = 0; i < len; ++i) {
        const double a = v[i];
        double* row = &c[(size_t)(lo + i) * r];
        for (int t2 = t + 1; t2 < r; ++t2) row[t2] -= a * sv[t2];
      }
    }
    // the right-hand sides
    for (int j = 0; j < J; ++j) sv[j] = 0.0;
    for (int i = 0; i < len; ++i) {
      const double a = v[i];
      const double* row = &g[(size_t)(lo + i) * J];
      for (int j = 0; j < J; ++j) sv[j] += a * row[j];
    }
    for (int j = 0; j < J; ++j) sv[j] *= tau;
    for (int i = 0; i < len; ++i) {
      const double a = v[i];
      double* row = &g[(size_t)(lo + i) * J];
      for (int j = 0; j < J; ++j) row[j] -= a * sv[j];
    }
  }
  for (int i = 0; i < (k + 1) * r; ++i)
    std::copy(&c[(size_t)i * r], &c[(size_t)i * r] + r, &R[(size_t)i * ldr + (size_t)k * r]);
  double dmax = 0.0;
  for (int i = 0; i < (k + 1) * r; ++i) dmax = std::max(dmax, std::fabs(R[(size_t)i * ldr + i]));
  for (int t = 0; t < r; ++t) {
    const double d = std::fabs(R[(size_t)(k * r + t) * ldr + k * r + t]);
    if (!(d > 1e-14 * dmax)) ok = false;
  }
  k++;
  return ok;
}

double BlockLS::resid(int j) const {
  double acc = 0.0;
  for (int i = k * r; i < (k + 1) * r; ++i) acc += g[(size_t)i * J + j] * g[(size_t)i * J + j];
  return std::sqrt(acc);
}

// Back substitution for all right-hand sides at once (inner loop over J).
void BlockLS::solve(std::vector<double>& Y) const {
  const int n = k * r;
  Y.assign((size_t)n * J, 0.0);
  for (int i = n - 1; i >= 0; --i) {
    double* y = &Y[(size_t)i * J];
    for (int j = 0; j < J; ++j) y[j] = g[(size_t)i * J + j];
    const double* Ri = &R[(size_t)i * ldr];
    for (int cc = i + 1; cc < n; ++cc) {
      const double a = Ri[cc];
      const double* yc = &Y[(size_t)cc * J];
      for (int j = 0; j < J; ++j) y[j] -= a * yc[j];
    }
    const double d = Ri[i];
    for (int j = 0; j < J; ++j) y[j] = (d != 0.0) ? y[j] / d : 0.0;
  }
}

}  // namespace mhde
