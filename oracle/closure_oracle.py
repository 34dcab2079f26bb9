"""Plain FP64 reference of the learned heat-flux closure's per-cell arithmetic (test
infrastructure only).

TEST INFRASTRUCTURE ONLY: imported by the test suite, the smoke check and the CPU-baseline leg
of the benchmark; the product path never uses it.  It shares no code with the CUDA library.

The closure is the library's extension (the paper has no learned closure).  For every spatial
cell it defines, from Q^n alone:

* the Chapman-Enskog heat flux H_CE: the velocity moments eps int c (x) c (x) c Ghat dv of the
  transport part of Ghat (Eq. 5-97) for the Maxwellian of the cell.  With p = rho T, the
  discrete temperature gradient (T_x, T_y) of Eq. (5-97more) and the Gaussian moments
  <c1^4> = 3T^2, <c1^6> = 15T^3, <c1^4 c2^2> = 3T^3 one finds
      H111 = -3 eps p T_x / tau,  H112 = -eps p T_y / tau,
      H122 = -eps p T_x / tau,    H222 = -3 eps p T_y / tau
  (the strain terms and (Gcal - M)/eps have no odd central moments);
* the scale s = eps rho T^{3/2} of the heat flux, and the network target
  y = (H - H_CE) / s, H being the heat flux of Eq. (5-99) from the micro step;
* 39 features: with the cell Knudsen number k = eps sqrt(T) / (tau h), h = min(dx, dy) (the
  relaxation length over the mesh width, which makes differences between neighbours
  resolution-independent), for the 8 neighbours of the 3x3 stencil (rows j-1, j, j+1, columns
  i-1, i, i+1, the centre skipped) k (rho_n/rho - 1), k (u1_n - u1)/sqrt(T), k (u2_n - u2)/sqrt(T),
  k (T_n/T - 1); then (theta11 - theta22)/(2T), theta12/T with theta = P/rho, u1/sqrt(T),
  u2/sqrt(T), log10 eps, the relaxation weight omega1 = eps / (eps + dt tau) of the micro step
  and log10 k.  A neighbour outside the box is the periodic image, or else the cell itself, with
  the normal velocity negated at a specular wall;
* the indicator max_m |y_m| of the network's prediction; a cell takes the closure when it is at
  most the threshold and the cell does not touch a non-periodic boundary.

A closure cell skips the micro update and keeps its g, which nothing reads unless a micro cell
needs it: the micro sweeps of a cell read g^n in its 3x3 block (the x sweep runs on the micro
cells and on their y neighbours, whose G* the y sweep reads, and reads the x neighbours of
those).  So at step n every cell in the 3x3 blocks of the micro cells whose g^n was not produced
by the micro update of step n-1 is first reset to the asymptotic-preserving limit Ghat(Q^n)
(Eq. 5-97): g is maintained exactly where it is read.
"""
from __future__ import annotations

import math

import numpy as np

from oracle import oracle as O

PERIODIC, SPECULAR = 0, 2
N_FEAT = 39


def _cell_prims(grid, params, Q):
    nx, ny = grid.nx, grid.ny
    Qf = np.asarray(Q, dtype=np.float64).reshape(6, ny * nx)
    out = np.zeros((ny * nx, 8))
    for c in range(nx * ny):
        out[c] = O.prims(params, Qf[:, c])
    return out.reshape(ny, nx, 8)  # rho, u1, u2, T, P11, P12, P22, tau


def _nb(i, d, n, bc_lo, bc_hi):
    """Index of the neighbour i + d along an axis of n cells, and whether it is a mirror image."""
    k = i + d
    if 0 <= k < n:
        return k, False
    bc = bc_lo if k < 0 else bc_hi
    if bc == PERIODIC:
        return k % n, False
    return i, bc == SPECULAR


def features(grid, params, Q, eps, dt):
    """Features X [ny*nx][39], H_CE [4][ny][nx] and scale [ny][nx] of every cell."""
    nx, ny = grid.nx, grid.ny
    dx = (grid.x1 - grid.x0) / nx
    dy = (grid.y1 - grid.y0) / ny
    P = _cell_prims(grid, params, Q)
    bc = params.bc
    X = np.zeros((ny, nx, N_FEAT))
    Hce = np.zeros((4, ny, nx))
    scale = np.zeros((ny, nx))
    for j in range(ny):
        for i in range(nx):
            rho, u1, u2, T, P11, P12, P22, tau = P[j, i]
            sT = math.sqrt(T)
            k = eps * sT / (tau * min(dx, dy))
            f = []
            for dj in (-1, 0, 1):
                nj, fy = _nb(j, dj, ny, bc[2], bc[3])
                for di in (-1, 0, 1):
                    if di == 0 and dj == 0:
                        continue
                    ni, fx = _nb(i, di, nx, bc[0], bc[1])
                    r, a1, a2, Tn = P[nj, ni, 0], P[nj, ni, 1], P[nj, ni, 2], P[nj, ni, 3]
                    if fx:
                        a1 = -a1
                    if fy:
                        a2 = -a2
                    f += [k * (r / rho - 1.0), k * (a1 - u1) / sT, k * (a2 - u2) / sT,
                          k * (Tn / T - 1.0)]
            f += [(P11 - P22) / (2.0 * rho * T), P12 / (rho * T), u1 / sT, u2 / sT,
                  math.log10(eps), eps / (eps + dt * tau), math.log10(k)]
            X[j, i] = f
            # discrete temperature gradient of Eq. (5-97more): face temperatures (T_nb + T)/2
            iL, _ = _nb(i, -1, nx, bc[0], bc[1])
            iR, _ = _nb(i, 1, nx, bc[0], bc[1])
            jB, _ = _nb(j, -1, ny, bc[2], bc[3])
            jT, _ = _nb(j, 1, ny, bc[2], bc[3])
            Tx = (0.5 * (P[j, iR, 3] + T) - 0.5 * (T + P[j, iL, 3])) / dx
            Ty = (0.5 * (P[jT, i, 3] + T) - 0.5 * (T + P[jB, i, 3])) / dy
            p = rho * T
            Hce[0, j, i] = -3.0 * eps * p * Tx / tau
            Hce[1, j, i] = -eps * p * Ty / tau
            Hce[2, j, i] = -eps * p * Tx / tau
            Hce[3, j, i] = -3.0 * eps * p * Ty / tau
            scale[j, i] = eps * rho * T ** 1.5
    return X.reshape(ny * nx, N_FEAT), Hce, scale


def targets(H, Hce, scale):
    """Network targets y [ny*nx][4] = (H - H_CE) / s."""
    y = (np.asarray(H) - Hce) / scale[None]
    return y.reshape(4, -1).T.copy()


def boundary_cells(grid, params):
    nx, ny = grid.nx, grid.ny
    b = np.zeros((ny, nx), dtype=bool)
    if params.bc[0] != PERIODIC:
        b[:, 0] = True
    if params.bc[1] != PERIODIC:
        b[:, nx - 1] = True
    if params.bc[2] != PERIODIC:
        b[0, :] = True
    if params.bc[3] != PERIODIC:
        b[ny - 1, :] = True
    return b


def decide(grid, params, y, Hce, scale, threshold):
    """Closure flags [ny][nx] and the closure heat flux H_CE + s y [4][ny][nx]."""
    ny, nx = grid.ny, grid.nx
    yc = np.asarray(y, dtype=np.float64).reshape(ny, nx, 4)
    ind = np.max(np.abs(yc), axis=2)
    flags = (ind <= threshold) & ~boundary_cells(grid, params)
    Hcl = Hce + scale[None] * np.moveaxis(yc, 2, 0)
    return flags, Hcl, ind


def _dilate(mask, axis, periodic):
    """Cells with a set neighbour along axis (or set themselves); periodic sides wrap."""
    out = mask.copy()
    n = mask.shape[axis]
    for d in (-1, 1):
        sh = np.roll(mask, d, axis=axis)
        if not periodic:
            idx = [slice(None)] * 2
            idx[axis] = 0 if d == 1 else n - 1
            sh[tuple(idx)] = False
        out |= sh
    return out


def needed_cells(grid, params, micro):
    """Cells whose g^n the micro sweeps of the micro cells read: their 3x3 blocks."""
    yp = params.bc[2] == PERIODIC
    xp = params.bc[0] == PERIODIC
    return _dilate(_dilate(micro, 0, yp), 1, xp)


def hybrid_run(grid, params, Q, G, dt, eps, y_of_features, threshold, nsteps=1, valid=None):
    """nsteps hybrid steps: per step the features of Q^n, the network's y (y_of_features(X) ->
    [n][4]), the closure decision, the refresh g^n = Ghat(Q^n) of needed cells whose g^n is not
    current, then the step with H = H_CE + s y in closure cells.  valid [ny][nx]: cells whose
    g is current at the start (default all).  Returns (Q, G, H, flags per step, indicator per
    step, refresh per step)."""
    valid = np.ones((grid.ny, grid.nx), dtype=bool) if valid is None else valid.copy()
    flags_all, ind_all, ref_all = [], [], []
    H = None
    for _ in range(nsteps):
        X, Hce, scale = features(grid, params, Q, eps, dt)
        y = y_of_features(X)
        flags, Hcl, ind = decide(grid, params, y, Hce, scale, threshold)
        micro = ~flags
        refresh = needed_cells(grid, params, micro) & ~valid
        Q, G, H = O.step_closure(grid, params, Q, G, dt, eps, flags, refresh, Hcl)
        valid = micro
        flags_all.append(flags)
        ind_all.append(ind)
        ref_all.append(refresh)
    return Q, G, H, flags_all, ind_all, ref_all
