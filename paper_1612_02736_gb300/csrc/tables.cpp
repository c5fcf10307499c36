// Host-side tables: reference-element operators (Sec. 3.1-3.4) and the box tree with its
// Gaussian node bookkeeping (Sec. 2, Sec. 4, Sec. 5.1).  Plain C++17, no CUDA calls.
#include <algorithm>
#include <cmath>
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

static void finish_tree(Tree& t) {
  // heights
  for (int b = (int)t.boxes.size() - 1; b >= 0; --b) {
    Box& bx = t.boxes[b];
    if (bx.child[0] >= 0)
      bx.height = 1 + std::max(t.boxes[bx.child[0]].height, t.boxes[bx.child[1]].height);
  }
  t.height = t.boxes.empty() ? 0 : t.boxes[0].height;
  // edges: canonical numbering, leaves in order, sides S, E, N, W
  const int nl = (int)t.leaves.size();
  t.leaf_edges.assign((size_t)4 * nl, -1);
  std::map<std::tuple<int, int, int>, int> key2edge;  // (orient, line, start)
  t.edge_owners.clear();
  for (int lf = 0; lf < nl; ++lf) {
    const Box& b = t.boxes[t.leaves[lf]];
    std::tuple<int, int, int> keys[4] = {
        {0, b.j0, b.i0}, {1, b.i1, b.j0}, {0, b.j1, b.i0}, {1, b.i0, b.j0}};
    for (int s = 0; s < 4; ++s) {
      auto it = key2edge.find(keys[s]);
      int e;
      if (it == key2edge.end()) {
        e = t.n_edges++;
        key2edge[keys[s]] = e;
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

int make_uniform_tree(double x0, double y0, double x1, double y1, int nx, int ny, Tree& t) {
  t = Tree();
  t.X0 = x0; t.Y0 = y0; t.X1 = x1; t.Y1 = y1;
  t.nx = nx; t.ny = ny;
  t.leaves.assign((size_t)nx * ny, -1);
  auto xs = [&](int i) { return x0 + (x1 - x0) * (double)i / (double)nx; };
  auto ys = [&](int j) { return y0 + (y1 - y0) * (double)j / (double)ny; };
  struct Q { int parent, i0, i1, j0, j1; };
  std::vector<Q> queue{{-1, 0, nx, 0, ny}};
  while (!queue.empty()) {
    std::vector<Q> nq;
    for (const Q& e : queue) {
      Box b;
      b.i0 = e.i0; b.i1 = e.i1; b.j0 = e.j0; b.j1 = e.j1;
      b.x0 = xs(e.i0); b.x1 = xs(e.i1); b.y0 = ys(e.j0); b.y1 = ys(e.j1);
      b.parent = e.parent;
      const int id = (int)t.boxes.size();
      t.boxes.push_back(b);
      if (e.parent >= 0) {
        Box& pb = t.boxes[e.parent];
        if (pb.child[0] < 0) pb.child[0] = id; else pb.child[1] = id;
      }
      const int wi = e.i1 - e.i0, wj = e.j1 - e.j0;
      if (wi == 1 && wj == 1) {
        t.boxes[id].leaf = e.j0 * nx + e.i0;
        t.leaves[(size_t)e.j0 * nx + e.i0] = id;
        continue;
      }
      if (wi >= wj) {  // vertical cut (ties vertical)
        const int im = e.i0 + wi / 2;
        nq.push_back({id, e.i0, im, e.j0, e.j1});
        nq.push_back({id, im, e.i1, e.j0, e.j1});
      } else {
        const int jm = e.j0 + wj / 2;
        nq.push_back({id, e.i0, e.i1, e.j0, jm});
        nq.push_back({id, e.i0, e.i1, jm, e.j1});
      }
    }
    queue.swap(nq);
  }
  finish_tree(t);
  return 0;
}

void build_node_sets(const Tree& t, int q, NodeSets& ns) {
  ns = NodeSets();
  ns.q = q;
  ns.n_gauss = t.n_edges * q;
  const int nb = (int)t.boxes.size();
  ns.ge.assign(nb, {});
  ns.J3.assign(nb, {});
  ns.n1.assign(nb, 0);
  for (int b = nb - 1; b >= 0; --b) {
    const Box& bx = t.boxes[b];
    if (bx.leaf >= 0) {
      std::vector<int>& ge = ns.ge[b];
      ge.reserve(4 * q);
      for (int s = 0; s < 4; ++s) {
        const int e = t.leaf_edges[(size_t)4 * bx.leaf + s];
        for (int k = 0; k < q; ++k) ge.push_back(e * q + k);
      }
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
    std::vector<int>& ge = ns.ge[b];
    ge = J1;
    ge.insert(ge.end(), J2.begin(), J2.end());
  }
  ns.boundary.clear();
  for (int e = 0; e < t.n_edges; ++e)
    if (t.edge_owners[(size_t)2 * e + 1] < 0)
      for (int k = 0; k < q; ++k) ns.boundary.push_back(e * q + k);
}

}  // namespace hps
