"""Box trees and Gaussian node bookkeeping (Sec. 2, Sec. 4, Sec. 5.1, Sec. 6).

Geometry is kept in integer units of the finest grid (base leaf size / 2^levels), so
edges compare exactly.  Trees:

* ``uniform_tree``: nx x ny equal leaves over a rectangle, built by recursive halving
  (Sec. 2): a box is cut across its longer side (in leaves); on a tie the cut is vertical
  unless ``tie='h'``.  The child on the west (vertical cut) or south (horizontal cut) is
  alpha, the other beta.
* ``mask_tree``: the leaves of an nx x ny grid of squares that a mask keeps (a union of
  squares such as the L-shaped domain).  The bisection skips empty halves, so a box with
  one non-empty half is that half's box.
* ``refine_tree``: local refinement (Sec. 6.1): at each level every leaf close to one of
  the points (distance d <= sqrt(2) l for a leaf of side 2 l) is split into 2 x 2 leaves;
  in the binary tree the old leaf becomes a refined parent: a vertical cut into W/E
  halves, each cut horizontally into S/N leaves.

Boxes are numbered breadth-first from the root (id 0), so a parent always has a smaller
id than its children (Algorithms 1-2 preamble).  Leaves are numbered by the lower-left
corner (y first, then x): row-major for uniform grids.

Gaussian nodes (Sec. 5.1): every leaf side is an edge segment with q Gauss-Legendre nodes;
a segment shared exactly by two leaves carries one set of nodes.  Global ids are handed
out segment by segment, visiting leaves in leaf order and their sides S, E, N, W, the q
ids of a segment ascending along it.  A box's exterior list I_ge is S,E,N,W for a leaf and
J1 followed by J2 for a parent (Sec. 4); J3 lists the shared nodes in alpha's order.

Refined parents (Sec. 6.3): after a refined parent is merged from its children, each side
that faces a leaf of the parent's own size (a neighbour, read as "same size and sharing
the whole side") is re-expressed on that neighbour's coarse segment: P_up interpolates the
coarse data to the fine nodes of the side (one degree q-1 polynomial through the coarse
Gauss nodes) and P_down interpolates fine data to the coarse nodes, each coarse node from
the fine segment that contains it, averaging the two one-sided values when it sits exactly
on the boundary between two fine segments (odd q).  Sides facing refined leaves, larger
leaves or the domain boundary keep their fine nodes (P = I).

This module is oracle code (test infrastructure); see ``oracle/__init__.py``.
"""
import numpy as np

from .spectral import SIDES, gauss_nodes, interp_matrix


class Box:
    def __init__(self, span):
        self.id = -1
        self.span = span          # (i0, i1, j0, j1) in finest-grid units
        self.rect = None          # (x0, y0, x1, y1)
        self.leaf = -1            # leaf index, or -1 for a parent
        self.children = None      # (alpha, beta) box ids
        self.parent = -1
        self.refined = False      # root of a 2 x 2 refinement of a former leaf
        self.ge = None            # exterior Gaussian node ids as seen by the parent (I_ge)
        self.ge_old = None        # exterior ids after the merge, before coarsening
        self.J1 = self.J2 = self.J3 = None
        self.Pup = self.Pdown = None  # refined parents with a coarsened side


class Tree:
    """A binary tree of boxes with Gaussian node numbering and refinement operators."""

    def __init__(self, root, q, origin, unit):
        self.q = q
        self.origin = origin      # (x0, y0)
        self.unit = unit          # (ux, uy): size of one finest-grid unit
        boxes, queue = [], [root]
        while queue:
            nq = []
            for b in queue:
                b.id = len(boxes)
                boxes.append(b)
                if b.children is not None:
                    for c in b.children:
                        c.parent = b.id
                    nq.extend(b.children)
            queue = nq
        for b in boxes:
            if b.children is not None:
                b.children = tuple(c.id for c in b.children)
            i0, i1, j0, j1 = b.span
            ox, oy = origin
            ux, uy = unit
            b.rect = (ox + i0 * ux, oy + j0 * uy, ox + i1 * ux, oy + j1 * uy)
        self.boxes = boxes
        lv = sorted((b for b in boxes if b.children is None), key=lambda b: (b.span[2], b.span[0]))
        self.leaves = []
        for k, b in enumerate(lv):
            b.leaf = k
            self.leaves.append(b.id)
        self._number_nodes()
        self._merge_sets()

    @property
    def n_leaves(self):
        return len(self.leaves)

    def leaf_rect(self, lf):
        return self.boxes[self.leaves[lf]].rect

    @staticmethod
    def _side_keys(span):
        i0, i1, j0, j1 = span
        return {"S": ("h", j0, i0, i1), "E": ("v", i1, j0, j1), "N": ("h", j1, i0, i1), "W": ("v", i0, j0, j1)}

    def _number_nodes(self):
        q = self.q
        seg_ids = {}
        owners = {}               # global id -> list of (leaf, position in leaf I_ge)
        nxt = 0
        for lf, bid in enumerate(self.leaves):
            b = self.boxes[bid]
            keys = self._side_keys(b.span)
            ge = []
            for s in SIDES:
                k = keys[s]
                if k not in seg_ids:
                    seg_ids[k] = list(range(nxt, nxt + q))
                    nxt += q
                ge.extend(seg_ids[k])
            b.ge = list(ge)
            b.ge_old = list(ge)
            for pos, g in enumerate(ge):
                owners.setdefault(g, []).append((lf, pos))
        self.n_gauss = nxt
        self.owners = owners
        self.segments = seg_ids
        self.node_seg = {}
        for k, ids in seg_ids.items():
            for i, g in enumerate(ids):
                self.node_seg[g] = (k, i)
        interior = sorted(g for g, o in owners.items() if len(o) == 2)
        self.interior = np.array(interior, dtype=np.int64)
        pairs = []
        for g in interior:
            (la, pa), (lb, pb) = owners[g]
            if SIDES[pa // q] in ("W", "S"):
                (la, pa), (lb, pb) = (lb, pb), (la, pa)
            pairs.append((la, pa, lb, pb))
        self.interior_pairs = np.array(pairs, dtype=np.int64).reshape(-1, 4)

    def _seg_points(self, key):
        """Running coordinates (along the segment) of its q Gauss nodes, and the
        segment's [lo, hi] in physical units."""
        orient, line, lo, hi = key
        u = self.unit[0] if orient == "h" else self.unit[1]
        o = self.origin[0] if orient == "h" else self.origin[1]
        a, b = o + lo * u, o + hi * u
        g = gauss_nodes(self.q)[0]
        return a + 0.5 * (b - a) * (g + 1.0), a, b

    def _coarsen(self, b):
        """Coarsen the sides of refined parent b that face a same-size leaf (Sec. 6.3)."""
        keys = self._side_keys(b.span)
        old = b.ge_old
        pos_old = {g: k for k, g in enumerate(old)}
        i0, i1, j0, j1 = b.span
        side_of = {}
        for g in old:
            key, _ = self.node_seg[g]
            orient, line = key[0], key[1]
            if orient == "h":
                side_of[g] = "S" if line == j0 else "N"
            else:
                side_of[g] = "W" if line == i0 else "E"
        coarse = {}
        for s in SIDES:
            k = keys[s]
            if k in self.segments:
                ids = self.segments[k]
                if not any(g in pos_old for g in ids):
                    coarse[s] = ids
        if not coarse:
            b.ge = list(old)
            return
        keep = [g for g in old if side_of[g] not in coarse]
        new = keep + [g for s in SIDES if s in coarse for g in coarse[s]]
        pos_new = {g: k for k, g in enumerate(new)}
        Pup = np.zeros((len(old), len(new)))
        Pdown = np.zeros((len(new), len(old)))
        for g in keep:
            Pup[pos_old[g], pos_new[g]] = 1.0
            Pdown[pos_new[g], pos_old[g]] = 1.0
        for s, cids in coarse.items():
            cpts, _, _ = self._seg_points(keys[s])
            fine = [g for g in old if side_of[g] == s]
            fpts = np.array([self._seg_points(self.node_seg[g][0])[0][self.node_seg[g][1]] for g in fine])
            Iu = interp_matrix(cpts, fpts)
            for r, g in enumerate(fine):
                Pup[pos_old[g], [pos_new[c] for c in cids]] = Iu[r]
            fsegs = sorted({self.node_seg[g][0] for g in fine}, key=lambda k: k[2])
            for r, c in enumerate(cids):
                t = cpts[r]
                hits = []
                for fk in fsegs:
                    fp, a, bb = self._seg_points(fk)
                    if a <= t <= bb:
                        hits.append((fk, fp))
                w = 1.0 / len(hits)
                for fk, fp in hits:
                    row = interp_matrix(fp, [t])[0]
                    for i, g in enumerate(self.segments[fk]):
                        Pdown[pos_new[c], pos_old[g]] += w * row[i]
        b.ge = new
        b.Pup, b.Pdown = Pup, Pdown

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
            b.ge_old = b.J1 + b.J2
            b.ge = list(b.ge_old)
            if b.refined:
                self._coarsen(b)
        self.boundary = np.array(sorted(self.boxes[0].ge), dtype=np.int64)
        self.slave = {}   # fine node -> (refined parent id, row in its ge_old)
        self.coarse_of = {}  # coarse node -> (refined parent id, row in its ge)
        for b in self.boxes:
            if b.Pup is not None:
                seto, setn = set(b.ge_old), set(b.ge)
                for k, g in enumerate(b.ge_old):
                    if g not in setn:
                        self.slave[g] = (b.id, k)
                for k, g in enumerate(b.ge):
                    if g not in seto:
                        self.coarse_of[g] = (b.id, k)

    def order_up(self):
        """Box ids so that children precede parents (reverse breadth-first order)."""
        return list(range(len(self.boxes) - 1, -1, -1))

    def gauss_points(self):
        """Coordinates of all Gaussian nodes, indexed by global id."""
        xy = np.zeros((self.n_gauss, 2))
        for key, ids in self.segments.items():
            pts, _, _ = self._seg_points(key)
            orient, line = key[0], key[1]
            if orient == "h":
                xy[ids, 0] = pts
                xy[ids, 1] = self.origin[1] + line * self.unit[1]
            else:
                xy[ids, 0] = self.origin[0] + line * self.unit[0]
                xy[ids, 1] = pts
        return xy


def _bisect(i0, i1, j0, j1, present, tie="v"):
    """Subtree of the leaf-unit region [i0,i1) x [j0,j1) restricted to present cells."""
    if not any(present(i, j) for j in range(j0, j1) for i in range(i0, i1)):
        return None
    wi, wj = i1 - i0, j1 - j0
    if wi == 1 and wj == 1:
        return Box((i0, i1, j0, j1))
    if wi > wj or (wi == wj and tie == "v"):
        im = i0 + wi // 2
        parts = (_bisect(i0, im, j0, j1, present, tie), _bisect(im, i1, j0, j1, present, tie))
    else:
        jm = j0 + wj // 2
        parts = (_bisect(i0, i1, j0, jm, present, tie), _bisect(i0, i1, jm, j1, present, tie))
    if parts[0] is None:
        return parts[1]
    if parts[1] is None:
        return parts[0]
    b = Box((min(parts[0].span[0], parts[1].span[0]), max(parts[0].span[1], parts[1].span[1]),
             min(parts[0].span[2], parts[1].span[2]), max(parts[0].span[3], parts[1].span[3])))
    b.children = parts
    return b


def uniform_tree(x0, y0, x1, y1, nx, ny, q, tie="v"):
    """The tree of Sec. 2 for nx x ny equal leaves over [x0,x1] x [y0,y1]."""
    root = _bisect(0, nx, 0, ny, lambda i, j: True, tie)
    return Tree(root, q, (x0, y0), ((x1 - x0) / nx, (y1 - y0) / ny))


def mask_tree(x0, y0, h, nx, ny, mask, q):
    """Leaves: the squares [x0 + i h, x0 + (i+1) h] x [y0 + j h, ...] with mask[j][i] set."""
    mask = np.asarray(mask, dtype=bool)
    root = _bisect(0, nx, 0, ny, lambda i, j: bool(mask[j, i]))
    return Tree(root, q, (x0, y0), (h, h))


def l_shape_tree(n, q):
    """The L-shaped domain [-1,1]^2 minus [0,1] x [-1,0] on a 2n x 2n grid of squares."""
    mask = np.ones((2 * n, 2 * n), dtype=bool)
    mask[:n, n:] = False
    return mask_tree(-1.0, -1.0, 1.0 / n, 2 * n, 2 * n, mask, q)


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


def refine_tree(tree, points, levels):
    """A new tree with `levels` rounds of refinement toward the points (Sec. 6.1)."""
    scale = 2 ** levels

    def copy(bid):
        b = tree.boxes[bid]
        i0, i1, j0, j1 = b.span
        nb = Box((i0 * scale, i1 * scale, j0 * scale, j1 * scale))
        nb.refined = b.refined
        if b.children is not None:
            nb.children = tuple(copy(c) for c in b.children)
        return nb

    root = copy(0)
    ux, uy = tree.unit[0] / scale, tree.unit[1] / scale
    ox, oy = tree.origin

    def rect(b):
        i0, i1, j0, j1 = b.span
        return (ox + i0 * ux, oy + j0 * uy, ox + i1 * ux, oy + j1 * uy)

    def leaves(b, out):
        if b.children is None:
            out.append(b)
        else:
            for c in b.children:
                leaves(c, out)
        return out

    for _ in range(levels):
        for b in leaves(root, []):
            if any(close_to(rect(b), x) for x in points):
                i0, i1, j0, j1 = b.span
                im, jm = (i0 + i1) // 2, (j0 + j1) // 2
                w, e = Box((i0, im, j0, j1)), Box((im, i1, j0, j1))
                w.children = (Box((i0, im, j0, jm)), Box((i0, im, jm, j1)))
                e.children = (Box((im, i1, j0, jm)), Box((im, i1, jm, j1)))
                b.children = (w, e)
                b.refined = True
    return Tree(root, tree.q, tree.origin, (ux, uy))
