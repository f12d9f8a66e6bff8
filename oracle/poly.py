"""ORACLE -- test infrastructure only (see oracle/__init__.py).

The polynomial-patch lens transport map of one path, FP64 numpy, written
from its definition.  It is the paper's factorised map (Sec. 4.2, Eq. 11:
an output f(x) where the validity mask g(x) = 1, nothing elsewhere) over
the symmetry-reduced input of Sec. 4.1 (Eq. 10), with the regressor f a
least-squares polynomial per patch fitted to traced rays:

  Reduced input of an entrance ray (x, y, d) at wavelength lambda (nm):
    slopes s = (d_x / d_z, d_y / d_z); r = |(x, y)|; (c, s_) = (x, y) / r,
    or (1, 0) at r = 0; rotated slopes p = c s_x + s_ s_y (radial) and
    q' = c s_y - s_ s_x (tangential); mirror m = -1 if q' < 0 else 1,
    q = |q'|; w = (1000 / lambda)^2 (um^-2, so a Cauchy index A + B w is
    affine in it).  u = (r, p, q, w) lies in the box
    [0, rho] x [-smax, smax] x [0, smax] x [(1000/lam_hi)^2, (1000/lam_lo)^2].
    The reduced ray is (x, y) = (r, 0), d = normalize(p, q, 1).
  Regressor f: the box is split into patches[k] equal patches per axis.
    On patch P the outputs (x', y', d_x', d_y', I) of the reduced ray are a
    polynomial of total degree <= D in the patch-local coordinates
    xi = 2 (u - lo_P) / h_P - 1 in [-1, 1]^4.  Its coefficients minimise the
    sum of squared errors over the patch's samples (a tensor grid of
    `samples` Chebyshev nodes cos(pi (k + 1/2) / samples) per axis) traced
    through the UNCLIPPED lens: the same surfaces and path with every clear
    aperture and the stop removed.  Apertures only decide validity; they do
    not change where a passing ray goes, so the unclipped transfer is the
    smooth function the valid rays follow, and the mask alone carries the
    occlusion (the paper's reason for factorising).  Samples lost anyway
    (a missed surface, TIR on a transmitted step) are left out of the sum; a
    patch with fewer valid samples than terms, or a rank-deficient design,
    has no fit.
  Mask g: the class grid has patches[k] * cells[k] cells per axis; its nodes
    u_i = lo + i * step (FP32 rule below) are traced through the REAL lens.
    A cell is INVALID if its 16 corner nodes are all invalid (and no fit ray
    inside it is valid), VALID if all 16 are valid, its patch has a fit, and
    every corner's (and every fit ray's) exit position is within
    max_residual_mm of the polynomial's, BOUNDARY otherwise.
  Query: VALID cell -> the polynomial at the ray's xi, d_z' = sqrt(1 - d_x'^2
    - d_y'^2), then mirrored (y', d_y' times m) and rotated back by (c, s_);
    INVALID -> no output; BOUNDARY or outside the box -> the exact tracer.

FP32 rule (shared by definition with the CUDA path, so both pick the same
cell for a ray on a face): the reduced coordinates and the class-grid
coordinate g_k = (u_k - lo_k) * inv_k are computed in FP32 with correctly
rounded operations in this order: i_z = 1 / d_z; s = d_xy * i_z; r2 = x*x +
y*y; r = sqrt(r2); i_r = 1 / r; c = x * i_r, s_ = y * i_r; p = c*s_x +
s_*s_y; q' = c*s_y - s_*s_x; t = 1000 / lambda; w = t*t; lo_k, step_k =
(hi_k - lo_k) / C_k and
inv_k = C_k / (hi_k - lo_k) are the FP32 roundings of the FP64 values;
cell_k = min(floor(g_k), C_k - 1), inside iff 0 <= g_k <= C_k.  Node rays:
v = lo + i * step; x = v_r; y = 0; n2 = (p*p + q*q) + 1; len = sqrt(n2);
d = (p / len, q / len, 1 / len); lambda = 1000 / sqrt(w).

Everything else (xi, the fit, the evaluation) is FP64.  Sample rays and
node rays are traced as FP32 inputs (the oracle tracer's interface).

Parity status: pinned -- exact reproduction of polynomial fields of degree
<= D and non-reproduction at D + 1, the reduction's round trip and
rotation invariance, the unclipped lens agreeing with the real lens on
every valid ray, brute-force classes from freshly traced corners, and the
map against the exact FP64 trace within its certified residual.
"""
from __future__ import annotations

import copy
import itertools
import math
from typing import Callable, Optional

import numpy as np

F32 = np.float32
CELL_INVALID, CELL_VALID, CELL_BOUNDARY = 0, 1, 2


def exponents(D: int):
    """Every exponent tuple (a, b, c, e) of (xi_r, xi_p, xi_q, xi_w) with
    a + b + c + e <= D."""
    return [t for t in itertools.product(range(D + 1), repeat=4) if sum(t) <= D]


def monomials(xi: np.ndarray, exps) -> np.ndarray:
    """Design matrix: row j, column t = prod_k xi[j, k] ** exps[t][k]."""
    xi = np.asarray(xi, np.float64)
    cols = [np.prod([xi[:, k] ** e[k] for k in range(4)], axis=0) for e in exps]
    return np.stack(cols, axis=1)


def reduce_f64(x, y, dx, dy, dz, lam):
    """FP64 reduced coordinates: (u [n,4], c, s, m)."""
    x, y, dx, dy, dz, lam = (np.asarray(a, np.float64) for a in (x, y, dx, dy, dz, lam))
    sx, sy = dx / dz, dy / dz
    r = np.sqrt(x * x + y * y)
    pos = r > 0
    rs = np.where(pos, r, 1.0)
    c = np.where(pos, x / rs, 1.0)
    s = np.where(pos, y / rs, 0.0)
    p = c * sx + s * sy
    qq = c * sy - s * sx
    m = np.where(qq < 0, -1.0, 1.0)
    w = (1000.0 / lam) ** 2
    return np.stack([r, p, np.abs(qq), w], axis=1), c, s, m


def reduce_f32(x, y, dx, dy, dz, lam):
    """The FP32 rule: reduced coordinates u [n,4] (float32), and whether the
    input is usable (finite, d_z > 0, lambda > 0)."""
    x, y, dx, dy, dz, lam = (np.asarray(a, F32) for a in (x, y, dx, dy, dz, lam))
    with np.errstate(all="ignore"):
        ok = (np.isfinite(x) & np.isfinite(y) & np.isfinite(dx) & np.isfinite(dy) & np.isfinite(dz)
              & np.isfinite(lam) & (dz > 0) & (lam > 0))
        idz = F32(1) / dz
        sx = dx * idz
        sy = dy * idz
        r2 = x * x + y * y
        r = np.sqrt(r2)
        pos = r > 0
        ir = F32(1) / np.where(pos, r, F32(1))
        c = np.where(pos, x * ir, F32(1)).astype(F32)
        s = np.where(pos, y * ir, F32(0)).astype(F32)
        p = c * sx + s * sy
        qq = c * sy - s * sx
        q = np.abs(qq)
        t = F32(1000) / lam
        w = t * t
    u = np.stack([r, p, q, w], axis=1).astype(F32)
    return u, ok


def reduced_rays_f64(u):
    """FP64 entrance rays (x, y, dx, dy, dz, lam) of reduced coordinates u [n,4]."""
    u = np.asarray(u, np.float64)
    r, p, q, w = u.T
    inv = 1.0 / np.sqrt(p * p + q * q + 1.0)
    return r, np.zeros_like(r), p * inv, q * inv, inv, 1000.0 / np.sqrt(w)


def unclipped(presc):
    """The prescription with every clear aperture and the stop removed (an
    even asphere keeps the edge of its conic's domain)."""
    U = copy.deepcopy(presc)
    for s in U.surfaces:
        a = 1e30
        kappa = float(getattr(s, "conic", 0.0))
        asph = tuple(getattr(s, "asph", (0.0, 0.0, 0.0, 0.0)))
        if kappa != 0.0 or any(v != 0.0 for v in asph):
            k2 = (1.0 + kappa) * s.curvature * s.curvature
            if k2 > 0:
                a = (1.0 - 1e-12) / math.sqrt(k2)
        s.aperture_r = a
    U.stop_r = 0.0
    return U


class PolyGrid:
    """Box, patch grid and class grid, with the FP32 constants of the rule."""

    def __init__(self, rho, smax, lam_lo, lam_hi, patches, cells):
        t_lo, t_hi = 1000.0 / lam_hi, 1000.0 / lam_lo
        self.lo = np.array([0.0, -smax, 0.0, t_lo * t_lo], np.float64)
        self.hi = np.array([rho, smax, smax, t_hi * t_hi], np.float64)
        self.P = np.asarray(patches, np.int64)
        self.m = np.asarray(cells, np.int64)
        self.C = self.P * self.m
        self.h = (self.hi - self.lo) / self.P          # patch sides (FP64)
        self.lo_f = self.lo.astype(F32)
        self.step_f = ((self.hi - self.lo) / self.C).astype(F32)
        self.inv_f = (self.C / (self.hi - self.lo)).astype(F32)

    @property
    def n_patches(self) -> int:
        return int(np.prod(self.P))

    @property
    def n_cells(self) -> int:
        return int(np.prod(self.C))

    def node_shape(self):
        return tuple(int(c) + 1 for c in self.C)

    def patch_lo(self, pidx):
        return self.lo + np.asarray(pidx, np.float64) * self.h

    def grid_coords(self, u32):
        """FP32 class-grid coordinates g [n,4] and inside [n]."""
        with np.errstate(all="ignore"):
            g = (np.asarray(u32, F32) - self.lo_f) * self.inv_f
        inside = np.all((g >= 0) & (g <= self.C.astype(F32)), axis=1)
        return g, inside

    def cell_of(self, g):
        """Class-grid cell index [n,4] of FP32 grid coordinates."""
        with np.errstate(all="ignore"):
            fl = np.floor(np.where(np.isfinite(g), g, 0)).astype(np.int64)
        return np.clip(fl, 0, self.C - 1)

    def node_rays_f32(self, idx):
        """FP32 entrance rays of class-grid nodes idx [n,4] (the FP32 rule)."""
        idx = np.asarray(idx, np.int64)
        v = (self.lo_f + idx.astype(F32) * self.step_f).astype(F32)
        r, p, q, w = v.T
        n2 = (p * p + q * q) + F32(1)
        ln = np.sqrt(n2)
        lam = F32(1000) / np.sqrt(w)
        return (r, np.zeros_like(r), (p / ln).astype(F32), (q / ln).astype(F32),
                (F32(1) / ln).astype(F32), lam.astype(F32))


def _rays(arrs):
    from paper_2605_04017_gb300.workloads import Rays
    return Rays(*[np.ascontiguousarray(a, F32) for a in arrs])


class PolyMap:
    """The oracle's own polynomial-patch map of one path, built from scratch."""

    def __init__(self, presc, path, rho, smax, lam_lo, lam_hi, degree, patches, cells, samples,
                 tol: float = float("inf"), fit_rays=None,
                 sample_fn: Optional[Callable] = None, node_fn: Optional[Callable] = None,
                 build_mask: bool = True):
        """sample_fn(u [n,4]) -> (values [n,5], valid [n]) replaces the
        unclipped trace of the fit samples, and node_fn(ray arrays) -> (out
        [n,6], valid [n]) the real trace of the class-grid nodes (the pins
        feed known fields through them).  build_mask False: no class table;
        classes come from classify_fresh, cell by cell (for maps too large to
        classify whole here)."""
        from oracle import Lens
        self.presc, self.path, self.tol, self.D = presc, tuple(path), float(tol), int(degree)
        self.lens = Lens(presc)
        self.open = Lens(unclipped(presc))
        self.grid = G = PolyGrid(rho, smax, lam_lo, lam_hi, patches, cells)
        self.exps = exponents(self.D)
        T = len(self.exps)
        ns = int(samples)
        cheb = np.cos(math.pi * (np.arange(ns) + 0.5) / ns)
        self.xi_s = np.array(list(itertools.product(cheb, repeat=4)), np.float64)
        A = monomials(self.xi_s, self.exps)
        if sample_fn is None:
            sample_fn = self._unclipped_samples
        # regressor: one least-squares fit per patch
        self.coef = np.zeros((G.n_patches, T, 5), np.float64)
        self.patch_ok = np.zeros(G.n_patches, bool)
        self.sample_res = np.zeros(G.n_patches, np.float64)
        for pid in range(G.n_patches):
            pidx = np.array(np.unravel_index(pid, tuple(G.P)))
            u = G.patch_lo(pidx) + (self.xi_s + 1.0) / 2.0 * G.h
            val, ok = sample_fn(u)
            if ok.sum() < T:
                continue
            Av = A[ok]
            if np.linalg.matrix_rank(Av) < T:
                continue
            c, *_ = np.linalg.lstsq(Av, val[ok], rcond=None)
            self.coef[pid] = c
            self.patch_ok[pid] = True
            self.sample_res[pid] = float(np.abs(Av @ c - val[ok]).max())
        self.fit_rays = fit_rays
        if not build_mask:
            return
        # mask: class-grid nodes through the real lens
        shape = G.node_shape()
        idx = np.array(list(np.ndindex(*shape)), np.int64)
        arrs = G.node_rays_f32(idx)
        if node_fn is None:
            out, v, _, _ = self.lens.trace(_rays(arrs), self.path)
            nv = v == 1
        else:
            out, nv = node_fn(arrs)
        self.node_out = out.reshape(shape + (6,))
        self.node_valid = nv.reshape(shape)
        self.cell_class, self.cell_res = self.classify_all()
        # fit rays: seen valid / invalid and residuals per cell
        if fit_rays is not None and len(fit_rays):
            self._apply_fit_rays(fit_rays)

    # -- regressor -----------------------------------------------------------------------

    def _unclipped_samples(self, u):
        arrs = [a.astype(F32) for a in reduced_rays_f64(u)]
        out, v, _, _ = self.open.trace(_rays(arrs), self.path)
        return out[:, [0, 1, 2, 3, 5]], v == 1

    def patch_of_cell(self, cell):
        return np.asarray(cell, np.int64) // self.grid.m

    def evaluate(self, pidx, xi):
        """Reduced-frame outputs (x', y', d_x', d_y', I) [n,5] of patch pidx at xi [n,4]."""
        pid = int(np.ravel_multi_index(tuple(np.asarray(pidx, np.int64)), tuple(self.grid.P)))
        return monomials(np.atleast_2d(xi), self.exps) @ self.coef[pid]

    def node_xi(self, cell, corner):
        """xi of corner `corner` (0/1 per axis) of `cell` in the cell's patch."""
        cell = np.asarray(cell, np.int64)
        node = cell + np.asarray(corner, np.int64)
        P = cell // self.grid.m
        return 2.0 * (node - P * self.grid.m) / self.grid.m - 1.0

    # -- mask ----------------------------------------------------------------------------

    def classify(self, cell):
        """(class, largest corner residual) of one class-grid cell."""
        corners = list(itertools.product((0, 1), repeat=4))
        vs = [bool(self.node_valid[tuple(np.asarray(cell) + k)]) for k in corners]
        if not any(vs):
            return CELL_INVALID, 0.0
        if not all(vs):
            return CELL_BOUNDARY, 0.0
        P = self.patch_of_cell(cell)
        pid = int(np.ravel_multi_index(tuple(P), tuple(self.grid.P)))
        if not self.patch_ok[pid]:
            return CELL_BOUNDARY, 0.0
        xi = np.array([self.node_xi(cell, k) for k in corners])
        pred = self.evaluate(P, xi)
        tr = np.array([self.node_out[tuple(np.asarray(cell) + k)] for k in corners])
        res = float(np.hypot(pred[:, 0] - tr[:, 0], pred[:, 1] - tr[:, 1]).max())
        return (CELL_VALID if res <= self.tol else CELL_BOUNDARY), res

    def classify_all(self):
        """classify() of every cell, a patch's cells at a time."""
        G = self.grid
        C = tuple(int(c) for c in G.C)
        corners = list(itertools.product((0, 1), repeat=4))
        nv = self.node_valid
        allv = np.ones(C, bool)
        anyv = np.zeros(C, bool)
        for k in corners:
            sl = tuple(slice(k[d], k[d] + C[d]) for d in range(4))
            allv &= nv[sl]
            anyv |= nv[sl]
        cls = np.where(allv, CELL_VALID, np.where(anyv, CELL_BOUNDARY, CELL_INVALID)).astype(np.uint8)
        res = np.zeros(C, np.float64)
        m = tuple(int(v) for v in G.m)
        for pid in range(G.n_patches):
            P = np.array(np.unravel_index(pid, tuple(G.P)), np.int64)
            sl = tuple(slice(P[d] * m[d], (P[d] + 1) * m[d]) for d in range(4))
            if not self.patch_ok[pid]:
                cls[sl] = np.where(cls[sl] == CELL_VALID, CELL_BOUNDARY, cls[sl])
                continue
            cells = np.array(list(np.ndindex(*m)), np.int64) + P * G.m
            cells = cells[allv[tuple(cells.T)]]
            if cells.size == 0:
                continue
            worst = np.zeros(len(cells))
            for k in corners:
                node = cells + np.asarray(k)
                xi = 2.0 * (node - P * G.m) / G.m - 1.0
                pred = self.evaluate(P, xi)
                tr = self.node_out[tuple(node.T)]
                worst = np.maximum(worst, np.hypot(pred[:, 0] - tr[:, 0], pred[:, 1] - tr[:, 1]))
            res[tuple(cells.T)] = worst
            cls[tuple(cells.T)] = np.where(worst <= self.tol, CELL_VALID, CELL_BOUNDARY)
        return cls, res

    def classify_fresh(self, cell):
        """(class, largest residual) of one cell from its 16 corner rays traced
        here and the map's fit rays that fall in it."""
        G = self.grid
        cell = np.asarray(cell, np.int64)
        corners = np.array(list(itertools.product((0, 1), repeat=4)), np.int64)
        arrs = G.node_rays_f32(cell + corners)
        out, v, _, _ = self.lens.trace(_rays(arrs), self.path)
        vs = v == 1
        if not vs.any():
            cls, res = CELL_INVALID, 0.0
        elif not vs.all():
            cls, res = CELL_BOUNDARY, 0.0
        else:
            P = cell // G.m
            pid = int(np.ravel_multi_index(tuple(P), tuple(G.P)))
            if not self.patch_ok[pid]:
                cls, res = CELL_BOUNDARY, 0.0
            else:
                xi = 2.0 * (cell + corners - P * G.m) / G.m - 1.0
                pred = self.evaluate(P, xi)
                res = float(np.hypot(pred[:, 0] - out[:, 0], pred[:, 1] - out[:, 1]).max())
                cls = CELL_VALID if res <= self.tol else CELL_BOUNDARY
        idx = self._fit_rays_in(cell)
        if idx.size and cls != CELL_BOUNDARY:
            sub = self.fit_rays.subset(idx)
            o, v, _, _ = self.lens.trace(sub, self.path)
            valid = v == 1
            if cls == CELL_INVALID and valid.any():
                cls = CELL_BOUNDARY
            elif cls == CELL_VALID:
                if not valid.all():
                    cls = CELL_BOUNDARY
                else:
                    pred = self.predict(sub, np.tile(cell, (idx.size, 1)), np.arange(idx.size))
                    for j in range(idx.size):
                        r = math.hypot(pred[j][0] - o[j, 0], pred[j][1] - o[j, 1])
                        res = max(res, r)
                    if res > self.tol:
                        cls = CELL_BOUNDARY
        return cls, res

    def _fit_rays_in(self, cell):
        """Indices of the fit rays inside `cell` (an index sorted by cell, built once)."""
        if self.fit_rays is None or not len(self.fit_rays):
            return np.zeros(0, np.int64)
        G = self.grid
        if not hasattr(self, "_fit_order"):
            u32, ok = reduce_f32(*self.fit_rays.arrays())
            g, inside = G.grid_coords(u32)
            cid = np.ravel_multi_index(tuple(G.cell_of(g).T), tuple(G.C))
            cid = np.where(inside & ok, cid, -1)
            self._fit_order = np.argsort(cid, kind="stable")
            self._fit_sorted = cid[self._fit_order]
        c = int(np.ravel_multi_index(tuple(np.asarray(cell, np.int64)), tuple(G.C)))
        a, b = np.searchsorted(self._fit_sorted, [c, c + 1])
        return np.sort(self._fit_order[a:b])

    def classify_cells(self, cells):
        """classify_fresh of many cells [k,4] at once (one trace of all their
        corners, a patch's polynomial evaluated for all its cells together):
        (classes [k], residuals [k])."""
        G = self.grid
        cells = np.asarray(cells, np.int64).reshape(-1, 4)
        k = len(cells)
        corners = np.array(list(itertools.product((0, 1), repeat=4)), np.int64)
        nodes = (cells[:, None, :] + corners[None, :, :]).reshape(-1, 4)
        arrs = G.node_rays_f32(nodes)
        out, v, _, _ = self.lens.trace(_rays(arrs), self.path)
        vs = (v == 1).reshape(k, 16)
        out = out.reshape(k, 16, 6)
        cls = np.where(vs.all(1), CELL_VALID, np.where(vs.any(1), CELL_BOUNDARY, CELL_INVALID)).astype(np.uint8)
        res = np.zeros(k)
        P = cells // G.m
        pid = np.ravel_multi_index(tuple(P.T), tuple(G.P))
        cls[(cls == CELL_VALID) & ~self.patch_ok[pid]] = CELL_BOUNDARY
        for q in np.unique(pid[cls == CELL_VALID]):
            sel = np.nonzero((pid == q) & (cls == CELL_VALID))[0]
            xi = (2.0 * (cells[sel][:, None, :] + corners[None] - P[sel][:, None, :] * G.m) / G.m - 1.0).reshape(-1, 4)
            pred = (monomials(xi, self.exps) @ self.coef[q]).reshape(len(sel), 16, 5)
            r = np.hypot(pred[:, :, 0] - out[sel, :, 0], pred[:, :, 1] - out[sel, :, 1]).max(1)
            res[sel] = r
            cls[sel[r > self.tol]] = CELL_BOUNDARY
        # fit rays inside the cells can only demote them (all of them traced
        # and evaluated at once; per cell: any valid ray demotes an INVALID
        # cell, any invalid ray or residual above tol a VALID one)
        if self.fit_rays is not None and len(self.fit_rays):
            self._fit_rays_in(cells[0])
            cid = np.ravel_multi_index(tuple(cells.T), tuple(G.C))
            a = np.searchsorted(self._fit_sorted, cid)
            b = np.searchsorted(self._fit_sorted, cid + 1)
            owner = np.repeat(np.arange(k), b - a)
            idx = np.concatenate([self._fit_order[x:y] for x, y in zip(a, b)]) if owner.size else \
                np.zeros(0, np.int64)
            keep = cls[owner] != CELL_BOUNDARY
            owner, idx = owner[keep], idx[keep]
            if idx.size:
                sub = self.fit_rays.subset(idx)
                o, v2, _, _ = self.lens.trace(sub, self.path)
                valid = v2 == 1
                seen_v = np.zeros(k, bool)
                seen_i = np.zeros(k, bool)
                np.logical_or.at(seen_v, owner, valid)
                np.logical_or.at(seen_i, owner, ~valid)
                cls[(cls == CELL_INVALID) & seen_v] = CELL_BOUNDARY
                vsel = np.nonzero((cls[owner] == CELL_VALID) & valid)[0]
                if vsel.size:
                    pred = self.predict(sub, cells[owner], vsel)
                    r = np.array([math.hypot(pred[int(j)][0] - o[j, 0], pred[int(j)][1] - o[j, 1]) for j in vsel])
                    np.maximum.at(res, owner[vsel], r)
                bad = (cls == CELL_VALID) & (seen_i | (res > self.tol))
                cls[bad] = CELL_BOUNDARY
        return cls, res

    def _apply_fit_rays(self, rays):
        G = self.grid
        u32, ok = reduce_f32(*rays.arrays())
        g, inside = G.grid_coords(u32)
        inside &= ok
        out, v, _, _ = self.lens.trace(rays, self.path)
        valid = v == 1
        cells = G.cell_of(g)
        pred = self.predict(rays, cells, np.nonzero(inside & valid)[0])
        for r in np.nonzero(inside)[0]:
            cell = tuple(cells[r])
            k = self.cell_class[cell]
            if valid[r]:
                if k == CELL_INVALID:
                    self.cell_class[cell] = CELL_BOUNDARY
                elif k == CELL_VALID:
                    res = math.hypot(pred[r][0] - out[r, 0], pred[r][1] - out[r, 1])
                    self.cell_res[cell] = max(self.cell_res[cell], res)
                    if res > self.tol:
                        self.cell_class[cell] = CELL_BOUNDARY
            elif k == CELL_VALID:
                self.cell_class[cell] = CELL_BOUNDARY

    # -- query ---------------------------------------------------------------------------

    def predict(self, rays, cells, idx):
        """Exit rays [len(idx), 6] from the regressor for rays idx (each in its
        cell's patch), as a dict {r: ray}."""
        idx = np.asarray(idx, np.int64)
        if idx.size == 0:
            return {}
        G = self.grid
        arrs = [np.asarray(a)[idx] for a in rays.arrays()]
        u, c, s, m = reduce_f64(*arrs)
        P = np.asarray(cells, np.int64)[idx] // G.m
        pid = np.ravel_multi_index(tuple(P.T), tuple(G.P))
        red = np.zeros((idx.size, 5))
        for q in np.unique(pid):
            sel = pid == q
            xi = 2.0 * (u[sel] - G.patch_lo(P[sel][0])) / G.h - 1.0
            red[sel] = monomials(xi, self.exps) @ self.coef[q]
        xp, yp, dxp, dyp, I = red.T
        dzp = np.sqrt(np.maximum(0.0, 1.0 - dxp * dxp - dyp * dyp))
        yp, dyp = m * yp, m * dyp
        out = np.stack([c * xp - s * yp, s * xp + c * yp, c * dxp - s * dyp, s * dxp + c * dyp,
                        dzp, I], axis=1)
        return {int(r): out[j] for j, r in enumerate(idx)}

    def locate(self, rays):
        """(inside [n], class-grid cells [n,4]) by the FP32 rule."""
        u32, ok = reduce_f32(*rays.arrays())
        g, inside = self.grid.grid_coords(u32)
        return inside & ok, self.grid.cell_of(g)

    def query(self, rays, use_mask: bool = True, classes=None):
        """(out [n,6], flags [n]): bit0 valid, bit3 bad input, bit4 answered by the
        exact tracer, bit5 outside the box.  use_mask False: every ray inside the
        box whose patch has a fit gets the regressor's answer (Fig. 6 ablation).
        classes: the rays' cell classes when the map holds no class table."""
        G = self.grid
        n = len(rays)
        inside, cells = self.locate(rays)
        cls = np.full(n, CELL_BOUNDARY, np.uint8)
        if classes is not None:
            cls[inside] = np.asarray(classes, np.uint8)[inside]
        else:
            cls[inside] = self.cell_class[tuple(cells[inside].T)]
        if not use_mask:
            pid = np.ravel_multi_index(tuple((cells // G.m).T), tuple(G.P))
            cls[inside] = np.where(self.patch_ok[pid[inside]], CELL_VALID, CELL_BOUNDARY)
        out = np.zeros((n, 6), np.float64)
        flags = np.zeros(n, np.uint8)
        flags[~inside] |= 32
        iv = np.nonzero(cls == CELL_VALID)[0]
        for r, o in self.predict(rays, cells, iv).items():
            out[r] = o
            flags[r] |= 1
        tr = np.nonzero(cls == CELL_BOUNDARY)[0]
        if tr.size:
            sub = rays.subset(tr)
            o, v, _, _ = self.lens.trace(sub, self.path)
            out[tr] = o
            flags[tr] |= 16 | np.where(v == 1, 1, 0).astype(np.uint8) | np.where(v == 8, 8, 0).astype(np.uint8)
        return out, flags
