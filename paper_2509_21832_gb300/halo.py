"""Spatial block decomposition of one micro-macro problem with face halos.

The paper's solver (Section 5.5) splits the spatial grid into 2D blocks, one per process, never
splits the velocity mesh, and exchanges face values of neighbouring blocks every step.  Here a
block is stepped as a problem of its own: its owned cells plus a halo of `w` cells on every side
that borders another block (or wraps around a periodic side), with extrapolation as a placeholder
rule beyond the halo.  One step changes a cell's Q through cells up to two away (the macro y
update reads Q* and H of its y neighbours, which read their x neighbours) and its g through cells
one away, so a halo of w >= 2 cells refreshed from the owners before every step gives every owned
cell bitwise the value of the undivided step: the arithmetic of every kernel for a cell depends
only on the values it reads, and the blocks are placed so that their cell sizes equal the
undivided grid's to the last bit.

`exchange` refreshes the halos point to point over torch.distributed (one process per block, any
backend, no collective); `exchange_local` does the same copies when every block lives in one
process.  Arrays are torch tensors (CPU or CUDA) or numpy arrays in the library's layouts:
Q [6][ny][nx] and G [ny][nx][nv2][nv1] of the block's extended grid.
"""
from dataclasses import dataclass, replace

import numpy as np

from . import inputs as I


@dataclass
class Block:
    rank: int
    bx: int
    by: int
    i0: int  # owned global cells [i0, i1) x [j0, j1)
    i1: int
    j0: int
    j1: int
    hl: int  # halo widths: left, right, bottom, top (0 where the block keeps a domain boundary)
    hr: int
    hb: int
    ht: int
    grid: I.Grid  # the extended block's grid (cell sizes bitwise those of the undivided grid)
    params: I.Params  # global boundary rules on kept domain sides, extrapolation beyond halos
    nx_glob: int
    ny_glob: int

    @property
    def nx(self):
        return self.i1 - self.i0 + self.hl + self.hr

    @property
    def ny(self):
        return self.j1 - self.j0 + self.hb + self.ht

    def global_index(self):
        """Global flat cell index (j nx + i) of every extended cell, [ny * nx] (periodic wrap)."""
        ii = (np.arange(self.i0 - self.hl, self.i1 + self.hr) % self.nx_glob)
        jj = (np.arange(self.j0 - self.hb, self.j1 + self.ht) % self.ny_glob)
        return (jj[:, None] * self.nx_glob + ii[None, :]).reshape(-1)

    def owned_mask(self):
        m = np.zeros((self.ny, self.nx), dtype=bool)
        m[self.hb:self.hb + self.j1 - self.j0, self.hl:self.hl + self.i1 - self.i0] = True
        return m.reshape(-1)

    def ext_index_of_owned(self, g):
        """Extended flat index of owned global cell(s) g."""
        g = np.asarray(g)
        i, j = g % self.nx_glob, g // self.nx_glob
        return (j - self.j0 + self.hb) * self.nx + (i - self.i0 + self.hl)


def _split(n, p):
    q, r = divmod(n, p)
    edges = [0]
    for k in range(p):
        edges.append(edges[-1] + q + (1 if k < r else 0))
    return edges


def _ulps(x, k):
    """x moved by k units in the last place (down for k < 0)."""
    for _ in range(abs(k)):
        x = np.nextafter(x, np.inf if k > 0 else -np.inf)
    return x


def _exact_extent(lo0, n, d, span=48):
    """(lo, hi) near (lo0, lo0 + n d) with (hi - lo) / n == d exactly (the library and the oracle
    both take the cell size as (hi - lo) / n; positions enter neither's plain step), or None: not
    every cell count admits one when d is not a dyadic fraction."""
    for a in range(2 * span + 1):
        lo = _ulps(lo0, (a + 1) // 2 * (1 if a % 2 else -1))  # lo0, +1, -1, +2, -2 ... ulps
        hi = lo + n * d
        for _ in range(span):
            q = (hi - lo) / n
            if q == d:
                return float(lo), float(hi)
            hi = np.nextafter(hi, np.inf if q < d else -np.inf)
    return None


def decompose(grid, params, px, py, w=2):
    """px x py blocks (rank = by px + bx) of the grid, each with halos of w cells."""
    if w < 2:
        raise ValueError("one step reads Q up to two cells away: the halo needs w >= 2")
    ex, ey = _split(grid.nx, px), _split(grid.ny, py)
    dx = (grid.x1 - grid.x0) / grid.nx
    dy = (grid.y1 - grid.y0) / grid.ny
    blocks = []
    for by in range(py):
        for bx in range(px):
            i0, i1, j0, j1 = ex[bx], ex[bx + 1], ey[by], ey[by + 1]
            if min(i1 - i0, j1 - j0) < w:
                raise ValueError("blocks need at least w owned cells per side")
            bc = list(params.bc)
            halo = [0, 0, 0, 0]
            for side, (first, last, p) in enumerate([(bx == 0, bx == px - 1, px)] * 2 +
                                                   [(by == 0, by == py - 1, py)] * 2):
                at_domain = first if side % 2 == 0 else last
                if p == 1:
                    continue  # the block spans the axis: the global rule on both sides
                if at_domain and params.bc[side] != I.PERIODIC:
                    continue  # a domain side with its own rule
                halo[side] = w
                bc[side] = I.EXTRAP  # placeholder beyond the halo
            # along each axis: the block's extent with the undivided cell size to the last bit;
            # where no extent of this cell count has it, one more halo cell at a time
            ext = []
            for (lo_side, hi_side, o0, o1, d, base) in ((0, 1, i0, i1, dx, grid.x0),
                                                        (2, 3, j0, j1, dy, grid.y0)):
                found = None
                for extra in range(8):
                    if extra and not (halo[lo_side] or halo[hi_side]):
                        break  # the block spans the axis with its own rules: nothing to widen
                    grow = hi_side if halo[hi_side] else lo_side
                    h = list(halo)
                    if extra:
                        h[grow] += extra
                    n = o1 - o0 + h[lo_side] + h[hi_side]
                    if not (halo[lo_side] or halo[hi_side]):
                        found = (h, (base, grid.x1 if lo_side == 0 else grid.y1))
                        break
                    lohi = _exact_extent(base + (o0 - h[lo_side]) * d, n, d)
                    if lohi is not None:
                        found = (h, lohi)
                        break
                if found is None:
                    raise ValueError("no block extent reproduces the cell size %r exactly" % d)
                halo[lo_side], halo[hi_side] = found[0][lo_side], found[0][hi_side]
                ext.append(found[1])
            hl, hr, hb, ht = halo
            nxe, nye = i1 - i0 + hl + hr, j1 - j0 + hb + ht
            (x0e, x1e), (y0e, y1e) = ext
            g = replace(grid, nx=nxe, ny=nye, x0=x0e, x1=x1e, y0=y0e, y1=y1e)
            assert (g.x1 - g.x0) / g.nx == dx and (g.y1 - g.y0) / g.ny == dy
            blocks.append(Block(by * px + bx, bx, by, i0, i1, j0, j1, hl, hr, hb, ht, g,
                                replace(params, bc=tuple(bc)), grid.nx, grid.ny))
    return blocks


def plan(blocks):
    """Point-to-point copies that refresh every halo: plan[(s, r)] = (src, dst), extended flat
    indices in block s (owned cells) and block r (halo cells), in the same order."""
    owner = np.empty(blocks[0].nx_glob * blocks[0].ny_glob, dtype=np.int64)
    for b in blocks:
        jj, ii = np.meshgrid(np.arange(b.j0, b.j1), np.arange(b.i0, b.i1), indexing="ij")
        owner[(jj * b.nx_glob + ii).reshape(-1)] = b.rank
    out = {}
    for r in blocks:
        gidx = r.global_index()
        halo = np.nonzero(~r.owned_mask())[0]
        for s in blocks:
            sel = halo[owner[gidx[halo]] == s.rank]
            if sel.size:
                out[(s.rank, r.rank)] = (s.ext_index_of_owned(gidx[sel]), sel)
    return out


def _flat(Q, G, b):
    """Views Q [6][ncell] and G [ncell][nv] of a block's extended arrays.  The arrays must be
    C-contiguous: a reshaped copy would take the halo writes and lose them."""
    nc = b.nx * b.ny
    for a in (Q, G):
        ok = a.is_contiguous() if hasattr(a, "is_contiguous") else a.flags["C_CONTIGUOUS"]
        if not ok:
            raise ValueError("block arrays must be C-contiguous (halo writes go through views)")
    if hasattr(Q, "is_contiguous"):      # torch: view() never copies
        return Q.view(6, nc), G.view(nc, -1)
    return Q.reshape(6, nc), G.reshape(nc, -1)   # C-contiguous numpy: reshape is a view


def scatter(blocks, Q, G):
    """Extended arrays of every block (owned cells and halos) from global arrays."""
    out = []
    nv = blocks[0].grid.nv1 * blocks[0].grid.nv2
    Qf, Gf = Q.reshape(6, -1), G.reshape(-1, nv)
    for b in blocks:
        gi = b.global_index()
        if hasattr(Q, "index_select"):
            import torch
            t = torch.as_tensor(gi, device=Q.device)
            Qb, Gb = Qf.index_select(1, t), Gf.index_select(0, t)
        else:
            Qb, Gb = Qf[:, gi], Gf[gi]
        out.append((Qb.reshape(6, b.ny, b.nx).contiguous() if hasattr(Qb, "contiguous")
                    else np.ascontiguousarray(Qb.reshape(6, b.ny, b.nx)),
                    Gb.reshape(b.ny, b.nx, b.grid.nv2, b.grid.nv1).contiguous()
                    if hasattr(Gb, "contiguous")
                    else np.ascontiguousarray(Gb.reshape(b.ny, b.nx, b.grid.nv2, b.grid.nv1))))
    return out


def gather(blocks, states, Q, G):
    """Write the owned cells of every block's (Q, G) into the global arrays Q, G."""
    nv = blocks[0].grid.nv1 * blocks[0].grid.nv2
    Qf, Gf = Q.reshape(6, -1), G.reshape(-1, nv)
    for b, (Qb, Gb) in zip(blocks, states):
        own = np.nonzero(b.owned_mask())[0]
        gi = b.global_index()[own]
        Qbf, Gbf = _flat(Qb, Gb, b)
        if hasattr(Q, "index_select"):
            import torch
            o = torch.as_tensor(own, device=Q.device)
            g = torch.as_tensor(gi, device=Q.device)
            Qf[:, g] = Qbf.index_select(1, o)
            Gf[g] = Gbf.index_select(0, o)
        else:
            Qf[:, gi] = Qbf[:, own]
            Gf[gi] = Gbf[own]


def exchange_local(blocks, copies, states):
    """Refresh every halo when all blocks live in one process (device-local copies)."""
    for (s, r), (src, dst) in sorted(copies.items()):
        Qs, Gs = _flat(*states[s], blocks[s])
        Qr, Gr = _flat(*states[r], blocks[r])
        if hasattr(Qs, "index_select"):
            import torch
            si = torch.as_tensor(src, device=Qs.device)
            di = torch.as_tensor(dst, device=Qs.device)
            Qr[:, di] = Qs.index_select(1, si)
            Gr[di] = Gs.index_select(0, si)
        else:
            Qr[:, dst] = Qs[:, src]
            Gr[dst] = Gs[src]


def exchange(blocks, copies, rank, Q, G, group=None):
    """Refresh the halos of block `rank` (torch tensors Q, G of its extended grid) from its
    neighbours and send them the cells they need: per neighbouring block one message of Q and one
    of g (each in its own dtype, so FP32 g travels as FP32) each way, all posted before any is
    waited on."""
    import torch
    import torch.distributed as dist
    b = blocks[rank]
    Qf, Gf = _flat(Q, G, b)
    nv = Gf.shape[1]
    reqs, recvs = [], []
    for (s, r), (src, dst) in sorted(copies.items()):
        if s == rank and r == rank:
            si = torch.as_tensor(src, device=Q.device)
            di = torch.as_tensor(dst, device=Q.device)
            Qf[:, di] = Qf.index_select(1, si)
            Gf[di] = Gf.index_select(0, si)
        elif s == rank:
            si = torch.as_tensor(src, device=Q.device)
            for msg in (Qf.index_select(1, si).contiguous(), Gf.index_select(0, si).contiguous()):
                reqs.append(dist.isend(msg, dst=r, group=group))
        elif r == rank:
            m = len(dst)
            qb = torch.empty((6, m), dtype=Q.dtype, device=Q.device)
            gb = torch.empty((m, nv), dtype=G.dtype, device=G.device)
            reqs.append(dist.irecv(qb, src=s, group=group))
            reqs.append(dist.irecv(gb, src=s, group=group))
            recvs.append((dst, qb, gb))
    for q in reqs:
        q.wait()
    for dst, qb, gb in recvs:
        di = torch.as_tensor(dst, device=Q.device)
        Qf[:, di] = qb
        Gf[di] = gb


def halo_regions(b):
    """The halo cells of block b as rectangles (i0, i1, j0, j1) of its extended grid."""
    out = []
    if b.hl:
        out.append((0, b.hl, 0, b.ny))
    if b.hr:
        out.append((b.nx - b.hr, b.nx, 0, b.ny))
    if b.hb:
        out.append((0, b.nx, 0, b.hb))
    if b.ht:
        out.append((0, b.nx, b.ny - b.ht, b.ny))
    return out


def block_shape(world):
    """px x py blocks for `world` ranks: the factorisation closest to square, px >= py."""
    py = max(p for p in range(1, int(world ** 0.5) + 1) if world % p == 0)
    return world // py, py
