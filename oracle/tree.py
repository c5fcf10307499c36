"""Box trees and Gaussian node bookkeeping (Sec. 2, Sec. 4, Sec. 5.1).

A uniform tree of nx x ny leaves over a rectangle is built by recursive halving (Sec. 2):
the box is cut across its longer side (in leaves); on a tie the cut is vertical unless
``tie='h'``.  The child on the west (cut vertical) or south (cut horizontal) is alpha,
the other is beta.  Boxes are numbered breadth-first from the root (id 0), so a parent
always has a smaller id than its children (Algorithm 1 and 2 preamble).

Gaussian nodes (Sec. 5.1): each leaf side carries q Gauss-Legendre nodes; a side shared
by two leaves carries one set of nodes.  Global ids are handed out edge by edge, visiting
leaves in leaf order (leaf = j * nx + i, x fastest) and their sides in the order S, E, N, W,
the q ids of an edge ascending along it.  A box's exterior list I_ge is S,E,N,W for a leaf
and J1 followed by J2 for a parent (Sec. 4); J3 lists the shared nodes in alpha's order.

This module is oracle code (test infrastructure); see ``oracle/__init__.py``.
"""
import numpy as np

from .spectral import SIDES


class Box:
    def __init__(self, bid, rect, span):
        self.id = bid
        self.rect = rect          # (x0, y0, x1, y1)
        self.span = span          # (i0, i1, j0, j1) in leaf units
        self.leaf = -1            # leaf index, or -1 for a parent
        self.children = None      # (alpha, beta) box ids
        self.parent = -1
        self.ge = None            # exterior Gaussian node ids (I_ge)
        self.J1 = self.J2 = self.J3 = None


class Tree:
    """A binary tree of boxes over a rectangle with Gaussian node numbering."""

    def __init__(self, boxes, leaves, nx, ny, q, rect):
        self.boxes = boxes
        self.leaves = leaves      # leaf index -> box id
        self.nx, self.ny, self.q, self.rect = nx, ny, q, rect
        self._number_nodes()
        self._merge_sets()

    @property
    def n_leaves(self):
        return len(self.leaves)

    def leaf_rect(self, lf):
        return self.boxes[self.leaves[lf]].rect

    def _number_nodes(self):
        q = self.q
        edge_ids = {}
        owners = {}               # global id -> list of (leaf, position in leaf I_ge)
        nxt = 0
        for lf, bid in enumerate(self.leaves):
            b = self.boxes[bid]
            i0, i1, j0, j1 = b.span
            keys = {"S": ("h", j0, i0), "E": ("v", i1, j0), "N": ("h", j1, i0), "W": ("v", i0, j0)}
            ge = []
            for s in SIDES:
                k = keys[s]
                if k not in edge_ids:
                    edge_ids[k] = list(range(nxt, nxt + q))
                    nxt += q
                ge.extend(edge_ids[k])
            b.ge = ge
            for pos, g in enumerate(ge):
                owners.setdefault(g, []).append((lf, pos))
        self.n_gauss = nxt
        self.owners = owners
        self.boundary = np.array(sorted(g for g, o in owners.items() if len(o) == 1), dtype=np.int64)
        interior = sorted(g for g, o in owners.items() if len(o) == 2)
        self.interior = np.array(interior, dtype=np.int64)
        # For each interior node: (leaf a, pos a, leaf b, pos b) with a the W (or S) leaf.
        pairs = []
        for g in interior:
            (la, pa), (lb, pb) = owners[g]
            side_a = SIDES[pa // q]
            if side_a in ("W", "S"):
                (la, pa), (lb, pb) = (lb, pb), (la, pa)
            pairs.append((la, pa, lb, pb))
        self.interior_pairs = np.array(pairs, dtype=np.int64).reshape(-1, 4)

    def _merge_sets(self):
        for bid in self.order_up():
            b = self.boxes[bid]
            if b.children is None:
                continue
            a, c = (self.boxes[k] for k in b.children)
            setb = set(c.ge)
            J3 = [g for g in a.ge if g in setb]
            set3 = set(J3)
            b.J3 = J3
            b.J1 = [g for g in a.ge if g not in set3]
            b.J2 = [g for g in c.ge if g not in set3]
            b.ge = b.J1 + b.J2

    def order_up(self):
        """Box ids so that children precede parents (reverse breadth-first order)."""
        return list(range(len(self.boxes) - 1, -1, -1))

    def gauss_points(self):
        """Coordinates of all Gaussian nodes, indexed by global id."""
        from .spectral import leaf_gauss_points
        xy = np.zeros((self.n_gauss, 2))
        for lf, bid in enumerate(self.leaves):
            b = self.boxes[bid]
            x0, y0, x1, y1 = b.rect
            gx, gy = leaf_gauss_points(x0, y0, x1 - x0, y1 - y0, self.q)
            xy[b.ge, 0] = gx
            xy[b.ge, 1] = gy
        return xy


def uniform_tree(x0, y0, x1, y1, nx, ny, q, tie="v"):
    """The tree of Sec. 2 for nx x ny equal leaves over [x0,x1] x [y0,y1]."""
    xs = [x0 + (x1 - x0) * i / nx for i in range(nx + 1)]
    ys = [y0 + (y1 - y0) * j / ny for j in range(ny + 1)]
    boxes = []
    leaves = [None] * (nx * ny)
    queue = [(-1, (0, nx, 0, ny))]
    while queue:
        nq = []
        for parent, span in queue:
            i0, i1, j0, j1 = span
            b = Box(len(boxes), (xs[i0], ys[j0], xs[i1], ys[j1]), span)
            b.parent = parent
            boxes.append(b)
            if parent >= 0:
                pb = boxes[parent]
                pb.children = (b.id,) if pb.children is None else pb.children + (b.id,)
            wi, wj = i1 - i0, j1 - j0
            if wi == 1 and wj == 1:
                b.leaf = j0 * nx + i0
                leaves[b.leaf] = b.id
                continue
            vertical = wi > wj or (wi == wj and tie == "v")
            if vertical:
                im = i0 + wi // 2
                nq += [(b.id, (i0, im, j0, j1)), (b.id, (im, i1, j0, j1))]
            else:
                jm = j0 + wj // 2
                nq += [(b.id, (i0, i1, j0, jm)), (b.id, (i0, i1, jm, j1))]
        queue = nq
    return Tree(boxes, leaves, nx, ny, q, (x0, y0, x1, y1))


def close_to(rect, xhat, t=np.sqrt(2.0)):
    """The closeness test of Sec. 6.1: a box of side 2 l is close to xhat when the distance
    d from xhat to the box satisfies d <= t l, with t = sqrt(2)."""
    x0, y0, x1, y1 = rect
    dx = max(x0 - xhat[0], 0.0, xhat[0] - x1)
    dy = max(y0 - xhat[1], 0.0, xhat[1] - y1)
    d = np.hypot(dx, dy)
    l = 0.5 * max(x1 - x0, y1 - y0)
    return d <= t * l


def refine_rects(rects, xhat, levels):
    """Sec. 6.1: at each refinement level, split every leaf that is close to xhat into a
    2 x 2 grid of equal leaves.  Returns the refined list of leaf rectangles."""
    rects = list(rects)
    for _ in range(levels):
        out = []
        for r in rects:
            if close_to(r, xhat):
                x0, y0, x1, y1 = r
                xm, ym = 0.5 * (x0 + x1), 0.5 * (y0 + y1)
                out += [(x0, y0, xm, ym), (xm, y0, x1, ym), (x0, ym, xm, y1), (xm, ym, x1, y1)]
            else:
                out.append(r)
        rects = out
    return rects
