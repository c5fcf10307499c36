// Host-side tables: reference-element operators (Sec. 3.1-3.4) and the box tree with its
// Gaussian node bookkeeping (Sec. 2, Sec. 4, Sec. 5.1).  Plain C++17, no CUDA calls.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <map>
#include <set>
#include <stdexcept>
#include <tuple>
#include <unordered_map>

#include "hps_internal.h"

namespace hps {

namespace {

const long double kPi = 3.141592653589793238462643383279502884L;

// Chebyshev-Lobatto points ascending: sin(pi (2k - N) / (2N)), N = p - 1 (the extrema of
// T_N, written in the symmetric sine form).
std::vector<double> lobatto(int p) {
  std::vector<double> x(p);
  const int N = p - 1;
  for (int k = 0; k < p; ++k) x[k] = (double)std::sin(kPi * (long double)(2 * k - N) / (2.0L * N));
  return x;
}

// Gauss-Legendre points ascending, by Newton's method on P_q with the three-term
// recurrence, started from the asymptotic guess cos(pi (k - 1/4) / (q + 1/2)).
std::vector<double> gauss_legendre(int q) {
  std::vector<double> x(q);
  for (int k = 1; k <= q; ++k) {
    long double z = std::cos(kPi * (k - 0.25L) / (q + 0.5L));
    for (int it = 0; it < 100; ++it) {
      long double p0 = 1.0L, p1 = z;
      for (int n = 2; n <= q; ++n) {
        long double p2 = ((2 * n - 1) * z * p1 - (n - 1) * p0) / n;
        p0 = p1;
        p1 = p2;
      }
      if (q == 1) { p1 = z; p0 = 1.0L; }
      long double dp = q * (z * p1 - p0) / (z * z - 1.0L);
      long double dz = p1 / dp;
      z -= dz;
      if (std::fabs((double)dz) < 1e-19) break;
    }
    x[q - k] = (double)z;  // cos guess descends in k -> store ascending
  }
  return x;
}

// Barycentric weights 1 / prod_{j != k}(x_k - x_j), accumulated in long double.
std::vector<long double> bary(const std::vector<double>& x) {
  const int n = (int)x.size();
  std::vector<long double> w(n);
  for (int k = 0; k < n; ++k) {
    long double prod = 1.0L;
    for (int j = 0; j < n; ++j)
      if (j != k) prod *= ((long double)x[k] - (long double)x[j]);
    w[k] = 1.0L / prod;
  }
  return w;
}

// Interpolation matrix (nt x ns, row-major) from nodes xs to targets xt (barycentric
// second form; a target equal to a node copies that node).
std::vector<double> interp(const std::vector<double>& xs, const std::vector<double>& xt) {
  const int ns = (int)xs.size(), nt = (int)xt.size();
  std::vector<long double> w = bary(xs);
  std::vector<double> P((size_t)nt * ns, 0.0);
  for (int i = 0; i < nt; ++i) {
    int hit = -1;
    for (int k = 0; k < ns; ++k)
      if (xt[i] == xs[k]) hit = k;
    if (hit >= 0) {
      P[(size_t)i * ns + hit] = 1.0;
      continue;
    }
    long double den = 0.0L;
    std::vector<long double> c(ns);
    for (int k = 0; k < ns; ++k) {
      c[k] = w[k] / ((long double)xt[i] - (long double)xs[k]);
      den += c[k];
    }
    for (int k = 0; k < ns; ++k) P[(size_t)i * ns + k] = (double)(c[k] / den);
  }
  return P;
}

// Chebyshev differentiation matrix on the ascending Lobatto points.  Off-diagonal entries
// from the explicit formula (c_i / c_j) (-1)^(i+j) / (x_i - x_j) with c = 2 at the ends;
// each diagonal entry is minus the sum of its row (exact on constants).
std::vector<double> cheb_diff(const std::vector<double>& x) {
  const int p = (int)x.size();
  std::vector<double> D((size_t)p * p, 0.0);
  for (int i = 0; i < p; ++i) {
    long double rs = 0.0L;
    const long double ci = (i == 0 || i == p - 1) ? 2.0L : 1.0L;
    for (int j = 0; j < p; ++j) {
      if (i == j) continue;
      const long double cj = (j == 0 || j == p - 1) ? 2.0L : 1.0L;
      const long double sgn = ((i + j) % 2) ? -1.0L : 1.0L;
      long double v = (ci / cj) * sgn / ((long double)x[i] - (long double)x[j]);
      D[(size_t)i * p + j] = (double)v;
      rs += v;
    }
    D[(size_t)i * p + i] = (double)(-rs);
  }
  return D;
}

}  // namespace

void build_ref_tables(int p, int q, RefTables& rt) {
  rt.p = p;
  rt.q = q;
  rt.m = (p - 2) * (p - 2);
  rt.ne = 4 * (p - 1);
  rt.xc = lobatto(p);
  rt.xg = gauss_legendre(q);
  rt.D = cheb_diff(rt.xc);
  rt.D2.assign((size_t)p * p, 0.0);
  for (int i = 0; i < p; ++i)
    for (int j = 0; j < p; ++j) {
      long double s = 0.0L;
      for (int k = 0; k < p; ++k) s += (long double)rt.D[i * p + k] * rt.D[k * p + j];
      rt.D2[i * p + j] = (double)s;
    }
  rt.Lg2c = interp(rt.xg, rt.xc);  // p x q
  rt.Lloc = interp(rt.xc, rt.xg);  // q x p
  rt.Ls = rt.Lg2c;
  for (int k = 0; k < q; ++k) {
    rt.Ls[0 * q + k] *= 0.5;
    rt.Ls[(size_t)(p - 1) * q + k] *= 0.5;
  }
  rt.DLs.assign((size_t)p * q, 0.0);
  for (int i = 0; i < p; ++i)
    for (int a = 0; a < q; ++a) {
      long double acc = 0.0L;
      for (int t = 0; t < p; ++t) acc += (long double)rt.D[(size_t)i * p + t] * rt.Ls[(size_t)t * q + a];
      rt.DLs[(size_t)i * q + a] = (double)acc;
    }
  rt.ci.clear();
  rt.ce.clear();
  for (int iy = 0; iy < p; ++iy)
    for (int ix = 0; ix < p; ++ix) {
      const bool ext = ix == 0 || ix == p - 1 || iy == 0 || iy == p - 1;
      (ext ? rt.ce : rt.ci).push_back(iy * p + ix);
    }
  // L_ce,ge (Eq. alpine2p5): each exterior node takes the side interpolant of every side
  // it lies on, with weight 1/(number of such sides) -- the corner average.
  const int nq = 4 * q;
  rt.Lce.assign((size_t)rt.ne * nq, 0.0);
  auto sides_of = [&](int node, int* sd, int* tt) {
    const int ix = node % p, iy = node / p;
    int n = 0;
    if (iy == 0) { sd[n] = 0; tt[n++] = ix; }
    if (ix == p - 1) { sd[n] = 1; tt[n++] = iy; }
    if (iy == p - 1) { sd[n] = 2; tt[n++] = ix; }
    if (ix == 0) { sd[n] = 3; tt[n++] = iy; }
    return n;
  };
  for (int e = 0; e < rt.ne; ++e) {
    int sd[2], tt[2];
    const int n = sides_of(rt.ce[e], sd, tt);
    for (int a = 0; a < n; ++a)
      for (int k = 0; k < q; ++k)
        rt.Lce[(size_t)e * nq + sd[a] * q + k] += rt.Lg2c[(size_t)tt[a] * q + k] / n;
  }
  // D_ge,c on [-1,1]^2 restricted to the exterior columns, then times L_ce,ge.
  // Row g = (side s, index a): S: Lloc[a][nx] D[0][ny]; E: Lloc[a][ny] D[p-1][nx];
  // N: Lloc[a][nx] D[p-1][ny]; W: Lloc[a][ny] D[0][nx]   (Sec. 3.4).
  auto dgec = [&](int s, int a, int node) -> double {
    const int nx = node % p, ny = node / p;
    switch (s) {
      case 0: return rt.Lloc[(size_t)a * p + nx] * rt.D[0 * p + ny];
      case 1: return rt.Lloc[(size_t)a * p + ny] * rt.D[(size_t)(p - 1) * p + nx];
      case 2: return rt.Lloc[(size_t)a * p + nx] * rt.D[(size_t)(p - 1) * p + ny];
      default: return rt.Lloc[(size_t)a * p + ny] * rt.D[0 * p + nx];
    }
  };
  rt.DceL.assign((size_t)nq * nq, 0.0);
  for (int s = 0; s < 4; ++s)
    for (int a = 0; a < q; ++a)
      for (int c = 0; c < nq; ++c) {
        long double acc = 0.0L;
        for (int e = 0; e < rt.ne; ++e) acc += (long double)dgec(s, a, rt.ce[e]) * rt.Lce[(size_t)e * nq + c];
        rt.DceL[(size_t)(s * q + a) * nq + c] = (double)acc;
      }
}

// ---------------------------------------------------------------------------------------
// Trees (Sec. 2, Sec. 6).  Geometry is in integer units of the finest grid, so edges
// compare exactly.  Trees are built as "proto" nodes, then numbered breadth-first.

namespace {

struct PNode {
  int i0, i1, j0, j1;
  int c0 = -1, c1 = -1;
  bool refined = false;
};

// Subtree of the cell region [i0,i1) x [j0,j1) restricted to present cells: the box is
// cut across its longer side (vertically on ties), empty halves are dropped.
int bisect(std::vector<PNode>& P, int i0, int i1, int j0, int j1, const std::vector<uint8_t>& present, int nx) {
  bool any = false;
  for (int j = j0; j < j1 && !any; ++j)
    for (int i = i0; i < i1; ++i)
      if (present[(size_t)j * nx + i]) {
        any = true;
        break;
      }
  if (!any) return -1;
  const int wi = i1 - i0, wj = j1 - j0;
  if (wi == 1 && wj == 1) {
    P.push_back(PNode{i0, i1, j0, j1});
    return (int)P.size() - 1;
  }
  int a, b;
  if (wi >= wj) {
    const int im = i0 + wi / 2;
    a = bisect(P, i0, im, j0, j1, present, nx);
    b = bisect(P, im, i1, j0, j1, present, nx);
  } else {
    const int jm = j0 + wj / 2;
    a = bisect(P, i0, i1, j0, jm, present, nx);
    b = bisect(P, i0, i1, jm, j1, present, nx);
  }
  if (a < 0) return b;
  if (b < 0) return a;
  PNode n{std::min(P[a].i0, P[b].i0), std::max(P[a].i1, P[b].i1), std::min(P[a].j0, P[b].j0),
          std::max(P[a].j1, P[b].j1)};
  n.c0 = a;
  n.c1 = b;
  P.push_back(n);
  return (int)P.size() - 1;
}

void finalize(const std::vector<PNode>& P, int root, double ox, double oy, double ux, double uy, Tree& t) {
  t = Tree();
  t.ox = ox;
  t.oy = oy;
  t.ux = ux;
  t.uy = uy;
  std::vector<int> map(P.size(), -1);
  std::vector<int> queue{root};
  std::vector<int> order;
  while (!queue.empty()) {
    std::vector<int> nq;
    for (int pi : queue) {
      map[pi] = (int)order.size();
      order.push_back(pi);
      if (P[pi].c0 >= 0) {
        nq.push_back(P[pi].c0);
        nq.push_back(P[pi].c1);
      }
    }
    queue.swap(nq);
  }
  t.boxes.resize(order.size());
  for (size_t k = 0; k < order.size(); ++k) {
    const PNode& n = P[order[k]];
    Box& b = t.boxes[k];
    b.i0 = n.i0; b.i1 = n.i1; b.j0 = n.j0; b.j1 = n.j1;
    b.x0 = ox + n.i0 * ux; b.x1 = ox + n.i1 * ux; b.y0 = oy + n.j0 * uy; b.y1 = oy + n.j1 * uy;
    b.refined = n.refined;
    if (n.c0 >= 0) {
      b.child[0] = map[n.c0];
      b.child[1] = map[n.c1];
      t.boxes[b.child[0]].parent = (int)k;
      t.boxes[b.child[1]].parent = (int)k;
    }
  }
  // heights
  for (int b = (int)t.boxes.size() - 1; b >= 0; --b) {
    Box& bx = t.boxes[b];
    if (bx.child[0] >= 0)
      bx.height = 1 + std::max(t.boxes[bx.child[0]].height, t.boxes[bx.child[1]].height);
  }
  t.height = t.boxes.empty() ? 0 : t.boxes[0].height;
  // leaves ordered by lower-left corner (y, then x): row-major on uniform grids
  for (size_t b = 0; b < t.boxes.size(); ++b)
    if (t.boxes[b].child[0] < 0) t.leaves.push_back((int)b);
  std::sort(t.leaves.begin(), t.leaves.end(), [&](int a, int b) {
    const Box &A = t.boxes[a], &B = t.boxes[b];
    return A.j0 != B.j0 ? A.j0 < B.j0 : A.i0 < B.i0;
  });
  for (size_t lf = 0; lf < t.leaves.size(); ++lf) t.boxes[t.leaves[lf]].leaf = (int)lf;
  // edge segments: canonical numbering, leaves in order, sides S, E, N, W
  const int nl = (int)t.leaves.size();
  t.leaf_edges.assign((size_t)4 * nl, -1);
  for (int lf = 0; lf < nl; ++lf) {
    const Box& b = t.boxes[t.leaves[lf]];
    const std::array<int, 4> keys[4] = {{0, b.j0, b.i0, b.i1}, {1, b.i1, b.j0, b.j1},
                                        {0, b.j1, b.i0, b.i1}, {1, b.i0, b.j0, b.j1}};
    for (int s = 0; s < 4; ++s) {
      auto it = t.edge_of.find(keys[s]);
      int e;
      if (it == t.edge_of.end()) {
        e = t.n_edges++;
        t.edge_of[keys[s]] = e;
        t.edge_keys.push_back(keys[s]);
        t.edge_owners.push_back(lf * 4 + s);
        t.edge_owners.push_back(-1);
      } else {
        e = it->second;
        t.edge_owners[(size_t)2 * e + 1] = lf * 4 + s;
      }
      t.leaf_edges[(size_t)4 * lf + s] = e;
    }
  }
}

void to_protos(const Tree& t, int b, int scale, std::vector<PNode>& P, std::vector<int>& idx) {
  const Box& bx = t.boxes[b];
  PNode n{bx.i0 * scale, bx.i1 * scale, bx.j0 * scale, bx.j1 * scale};
  n.refined = bx.refined;
  P.push_back(n);
  const int me = (int)P.size() - 1;
  idx[b] = me;
  if (bx.child[0] >= 0) {
    to_protos(t, bx.child[0], scale, P, idx);
    to_protos(t, bx.child[1], scale, P, idx);
    P[me].c0 = idx[bx.child[0]];
    P[me].c1 = idx[bx.child[1]];
  }
}

}  // namespace

int make_uniform_tree(double x0, double y0, double x1, double y1, int nx, int ny, Tree& t) {
  std::vector<uint8_t> all((size_t)nx * ny, 1);
  std::vector<PNode> P;
  const int root = bisect(P, 0, nx, 0, ny, all, nx);
  finalize(P, root, x0, y0, (x1 - x0) / nx, (y1 - y0) / ny, t);
  return 0;
}

int make_mask_tree(double x0, double y0, double h, int nx, int ny, const uint8_t* mask, Tree& t) {
  std::vector<uint8_t> present(mask, mask + (size_t)nx * ny);
  std::vector<PNode> P;
  const int root = bisect(P, 0, nx, 0, ny, present, nx);
  if (root < 0) return 1;
  finalize(P, root, x0, y0, h, h, t);
  return 0;
}

// Sec. 6.1: at each level every leaf whose distance d to one of the points satisfies
// d <= sqrt(2) l (side 2 l) is split 2 x 2: a vertical cut into W/E halves, each cut
// horizontally into S/N leaves; the former leaf is marked as a refined parent.
int refine_tree(const Tree& in, const double* pts, int npts, int levels, Tree& out) {
  const int scale = 1 << levels;
  std::vector<PNode> P;
  std::vector<int> idx(in.boxes.size(), -1);
  to_protos(in, 0, scale, P, idx);
  const double ux = in.ux / scale, uy = in.uy / scale;
  for (int lev = 0; lev < levels; ++lev) {
    const size_t n0 = P.size();
    for (size_t k = 0; k < n0; ++k) {
      if (P[k].c0 >= 0) continue;
      const double bx0 = in.ox + P[k].i0 * ux, bx1 = in.ox + P[k].i1 * ux;
      const double by0 = in.oy + P[k].j0 * uy, by1 = in.oy + P[k].j1 * uy;
      const double l = 0.5 * std::max(bx1 - bx0, by1 - by0);
      bool close = false;
      for (int pi = 0; pi < npts && !close; ++pi) {
        const double dx = std::max(std::max(bx0 - pts[2 * pi], 0.0), pts[2 * pi] - bx1);
        const double dy = std::max(std::max(by0 - pts[2 * pi + 1], 0.0), pts[2 * pi + 1] - by1);
        close = std::hypot(dx, dy) <= std::sqrt(2.0) * l;
      }
      if (!close) continue;
      const int i0 = P[k].i0, i1 = P[k].i1, j0 = P[k].j0, j1 = P[k].j1;
      const int im = (i0 + i1) / 2, jm = (j0 + j1) / 2;
      const int base = (int)P.size();
      P.push_back(PNode{i0, im, j0, jm});  // W-S
      P.push_back(PNode{i0, im, jm, j1});  // W-N
      P.push_back(PNode{im, i1, j0, jm});  // E-S
      P.push_back(PNode{im, i1, jm, j1});  // E-N
      PNode w{i0, im, j0, j1}, e{im, i1, j0, j1};
      w.c0 = base; w.c1 = base + 1;
      e.c0 = base + 2; e.c1 = base + 3;
      P.push_back(w);
      P.push_back(e);
      P[k].c0 = base + 4;
      P[k].c1 = base + 5;
      P[k].refined = true;
    }
  }
  finalize(P, 0, in.ox, in.oy, ux, uy, out);
  return 0;
}

void build_node_sets(const Tree& t, int q, NodeSets& ns, const std::vector<double>& xg) {
  ns = NodeSets();
  ns.q = q;
  ns.n_gauss = t.n_edges * q;
  const int nb = (int)t.boxes.size();
  ns.ge.assign(nb, {});
  ns.ge_old.assign(nb, {});
  ns.J3.assign(nb, {});
  ns.n1.assign(nb, 0);
  ns.co.assign(nb, Coarsen());
  // position of node (edge e, index k) along its segment, in physical units
  auto pos_along = [&](int node) {
    const std::array<int, 4>& key = t.edge_keys[node / q];
    const double u = key[0] == 0 ? t.ux : t.uy;
    const double o = key[0] == 0 ? t.ox : t.oy;
    const double a = o + key[2] * u, b = o + key[3] * u;
    return a + 0.5 * (b - a) * (xg[node % q] + 1.0);
  };
  for (int b = nb - 1; b >= 0; --b) {
    const Box& bx = t.boxes[b];
    if (bx.leaf >= 0) {
      std::vector<int>& ge = ns.ge[b];
      for (int s = 0; s < 4; ++s) {
        const int e = t.leaf_edges[(size_t)4 * bx.leaf + s];
        for (int k = 0; k < q; ++k) ge.push_back(e * q + k);
      }
      ns.ge_old[b] = ge;
      continue;
    }
    const std::vector<int>& ga = ns.ge[bx.child[0]];
    const std::vector<int>& gb = ns.ge[bx.child[1]];
    std::unordered_map<int, int> inb;
    inb.reserve(gb.size() * 2);
    for (size_t k = 0; k < gb.size(); ++k) inb[gb[k]] = (int)k;
    std::vector<int> J1, J3, J2;
    std::set<int> s3;
    for (int g : ga) {
      if (inb.count(g)) { J3.push_back(g); s3.insert(g); } else J1.push_back(g);
    }
    for (int g : gb)
      if (!s3.count(g)) J2.push_back(g);
    ns.J3[b] = J3;
    ns.n1[b] = (int)J1.size();
    std::vector<int>& old = ns.ge_old[b];
    old = J1;
    old.insert(old.end(), J2.begin(), J2.end());
    ns.ge[b] = old;
    if (!bx.refined) continue;
    // Sec. 6.3: coarsen every side that faces a leaf of this box's size
    std::set<int> inold(old.begin(), old.end());
    const std::array<int, 4> keys[4] = {{0, bx.j0, bx.i0, bx.i1}, {1, bx.i1, bx.j0, bx.j1},
                                        {0, bx.j1, bx.i0, bx.i1}, {1, bx.i0, bx.j0, bx.j1}};
    std::vector<int> cseg(4, -1);
    for (int s = 0; s < 4; ++s) {
      auto it = t.edge_of.find(keys[s]);
      if (it == t.edge_of.end()) continue;
      bool mine = false;
      for (int k = 0; k < q; ++k) mine = mine || inold.count(it->second * q + k);
      if (!mine) cseg[s] = it->second;
    }
    if (cseg[0] < 0 && cseg[1] < 0 && cseg[2] < 0 && cseg[3] < 0) continue;
    auto side_of = [&](int node) {
      const std::array<int, 4>& key = t.edge_keys[node / q];
      if (key[0] == 0) return key[1] == bx.j0 ? 0 : 2;
      return key[1] == bx.i1 ? 1 : 3;
    };
    Coarsen& C = ns.co[b];
    std::vector<int> nw;
    for (int g : old)
      if (cseg[side_of(g)] < 0) nw.push_back(g);
    for (int s = 0; s < 4; ++s)
      if (cseg[s] >= 0)
        for (int k = 0; k < q; ++k) nw.push_back(cseg[s] * q + k);
    std::unordered_map<int, int> po, pn;
    for (size_t k = 0; k < old.size(); ++k) po[old[k]] = (int)k;
    for (size_t k = 0; k < nw.size(); ++k) pn[nw[k]] = (int)k;
    const int ko = (int)old.size(), kn = (int)nw.size();
    C.Pup.assign((size_t)ko * kn, 0.0);
    C.Pdown.assign((size_t)kn * ko, 0.0);
    for (int g : old)
      if (cseg[side_of(g)] < 0) {
        C.Pup[(size_t)po[g] * kn + pn[g]] = 1.0;
        C.Pdown[(size_t)pn[g] * ko + po[g]] = 1.0;
      }
    for (int s = 0; s < 4; ++s) {
      if (cseg[s] < 0) continue;
      std::vector<double> cpts(q);
      for (int k = 0; k < q; ++k) cpts[k] = pos_along(cseg[s] * q + k);
      std::vector<int> fine;
      for (int g : old)
        if (side_of(g) == s) fine.push_back(g);
      // P_up: every fine node from the one polynomial through the coarse nodes
      std::vector<double> fpts;
      for (int g : fine) fpts.push_back(pos_along(g));
      const std::vector<double> Iu = interp(cpts, fpts);
      for (size_t r = 0; r < fine.size(); ++r)
        for (int k = 0; k < q; ++k) C.Pup[(size_t)po[fine[r]] * kn + pn[cseg[s] * q + k]] = Iu[r * q + k];
      // P_down: every coarse node from the fine segment(s) containing it (mean on a shared end)
      std::vector<int> fsegs;
      for (int g : fine)
        if (std::find(fsegs.begin(), fsegs.end(), g / q) == fsegs.end()) fsegs.push_back(g / q);
      for (int k = 0; k < q; ++k) {
        const double tc = cpts[k];
        std::vector<int> hits;
        for (int e : fsegs) {
          const std::array<int, 4>& key = t.edge_keys[e];
          const double u = key[0] == 0 ? t.ux : t.uy, o = key[0] == 0 ? t.ox : t.oy;
          if (o + key[2] * u <= tc && tc <= o + key[3] * u) hits.push_back(e);
        }
        for (int e : hits) {
          std::vector<double> fp(q);
          for (int i = 0; i < q; ++i) fp[i] = pos_along(e * q + i);
          const std::vector<double> row = interp(fp, std::vector<double>{tc});
          for (int i = 0; i < q; ++i)
            C.Pdown[(size_t)pn[cseg[s] * q + k] * ko + po[e * q + i]] += row[i] / (double)hits.size();
        }
      }
      for (int g : fine) C.fine.push_back(g);
      for (int k = 0; k < q; ++k) C.coarse.push_back(cseg[s] * q + k);
    }
    // rows of P_up for the fine nodes, columns for the coarse nodes
    const int nf = (int)C.fine.size(), nc = (int)C.coarse.size();
    C.Pupc.assign((size_t)nf * nc, 0.0);
    for (int r = 0; r < nf; ++r)
      for (int c = 0; c < nc; ++c) C.Pupc[(size_t)r * nc + c] = C.Pup[(size_t)po[C.fine[r]] * kn + pn[C.coarse[c]]];
    ns.ge[b] = nw;
    C.active = true;
  }
  ns.boundary = ns.ge[0];
  std::sort(ns.boundary.begin(), ns.boundary.end());
}

}  // namespace hps
