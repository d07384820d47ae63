"""Domain decomposition with halo exchange (paper Sec. 3.3), as contexts of
the library that hold parts of one grid.

The grid (nz, ny, nx) is split into px x py x pz owned boxes -- the paper's
slab-z (1, 1, 4), block-xy (2, 2, 1) and pencil-yz (1, 2, 2) layouts, or any
other.  Each part is one library context holding its owned box plus ghost
layers of depth g = 2 r s = 8 s in the decomposed directions (r = 4, the
radius of the stencil; a full step reaches 2 r nodes).  The CPML sits on the
grid's outer faces only: a part's face carries the global layer where it is a
grid face and none where it is an internal interface.  Every s steps the ghost
layers are refreshed from the parts that own those nodes (fdtd_exchange copies
p, v and the memory variables), and then every part advances s steps; the
owned boxes then hold exactly the values of one undivided grid (s = 1 is the
standard exchange, s > 1 the enlarged ghost region, Tab. 12).

Here all parts share one GPU, each on a stream of its own, so the exchange
kernel reads the neighbour's memory directly and the parts' steps run side by
side as they would on separate GPUs.  Events order the phases: every part
finishes its steps before any exchange reads it, and every exchange finishes
before any part steps again (the parts update their pressure memory variables
in place).
Sources are injected by every part whose box (ghosts included) contains them,
so that the ghost layers evolve as the grid does between exchanges; receivers
are recorded by their owner only.  This module does argument marshalling:
every step and every exchange runs in the library's kernels.
"""
from __future__ import annotations

import ctypes

import torch

from .fdtd import Fdtd, _cells6

RADIUS = 4


def split(n: int, parts: int):
    """Owned ranges [a, b) of `parts` near-equal pieces of n nodes."""
    base, extra = divmod(n, parts)
    out, a = [], 0
    for k in range(parts):
        b = a + base + (1 if k < extra else 0)
        out.append((a, b))
        a = b
    return out


def plan(shape, parts, s, cells):
    """Geometry of a decomposition: for each part (x fastest, then y, then
    z) its owned box and local box (owned plus ghosts of depth g = 8 s in the
    decomposed directions, clipped to the grid), as ((z0, z1), (y0, y1),
    (x0, x1)) in grid coordinates, and its CPML cells per face (the grid's
    where the local box reaches a grid face, 0 at an interface); and the
    links (i, j, box, shift): part i's ghost box, in its local coordinates,
    that part j owns, with the offset of j's local coordinates.  Raises if a
    part is too thin (its owned extent along a decomposed axis must reach
    g plus the layer's cells)."""
    nz, ny, nx = shape
    px, py, pz = parts
    g = 2 * RADIUS * s
    cells = _cells6(cells)
    rx, ry, rz = split(nx, px), split(ny, py), split(nz, pz)
    out = []
    for (z0, z1) in rz:
        for (y0, y1) in ry:
            for (x0, x1) in rx:
                own = ((z0, z1), (y0, y1), (x0, x1))
                loc = tuple((max(0, lo - (g if p > 1 else 0)), min(n, hi + (g if p > 1 else 0)))
                            for (lo, hi), n, p in zip(own, (nz, ny, nx), (pz, py, px)))
                c = list(cells)
                for axis, (lo, hi), n, p in ((0, own[2], nx, px), (1, own[1], ny, py), (2, own[0], nz, pz)):
                    llo, lhi = loc[2 - axis]
                    if llo > 0:
                        c[2 * axis] = 0
                    if lhi < n:
                        c[2 * axis + 1] = 0
                    need = g + max(cells[2 * axis:2 * axis + 2])
                    if p > 1 and hi - lo < need:
                        raise ValueError(f"a part spans {hi - lo} nodes along axis {'xyz'[axis]}: at least "
                                         f"g + cells = {need} needed")
                out.append(dict(own=own, loc=loc, cells=tuple(c)))
    links = []
    for i, a in enumerate(out):
        for j, b in enumerate(out):
            if i == j:
                continue
            box = []
            for ax in range(3):
                lo = max(a["loc"][ax][0], b["own"][ax][0])
                hi = min(a["loc"][ax][1], b["own"][ax][1])
                if lo >= hi:
                    break
                box += [lo - a["loc"][ax][0], hi - a["loc"][ax][0]]
            else:
                links.append((i, j, tuple(box), tuple(a["loc"][ax][0] - b["loc"][ax][0] for ax in range(3))))
    return out, links


class Decomposition:
    """A grid of shape (nz, ny, nx) split into parts = (px, py, pz) pieces
    along (x, y, z), exchanging ghosts of depth 8 s every s steps."""

    def __init__(self, shape, h, dt, parts=(1, 2, 2), s=1, *, nshots=1, cpml_cells=0, storage="f32", nt_max=1,
                 nrec_max=0, cpml_local=False, device=None, stream=None):
        self.shape = tuple(int(v) for v in shape)
        self.parts = tuple(int(p) for p in parts)
        self.s = int(s)
        if self.s < 1:
            raise ValueError("s must be >= 1")
        self.g = 2 * RADIUS * self.s
        self.cells = _cells6(cpml_cells)
        self.nshots, self.nt_max = int(nshots), int(nt_max)
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.stream = stream or torch.cuda.current_stream(self.device)
        geo, links = plan(self.shape, self.parts, self.s, self.cells)
        self.subs = []
        for part in geo:
            lshape = tuple(hi - lo for lo, hi in part["loc"])
            st = torch.cuda.Stream(self.device)
            sim = Fdtd(lshape, h, dt, nshots=self.nshots, cpml_cells=part["cells"], storage=storage,
                       nt_max=self.nt_max, nrec_max=nrec_max, cpml_local=cpml_local, device=self.device,
                       stream=st)
            self.subs.append(dict(sim=sim, stream=st, own=part["own"], loc=part["loc"], rec_cols=None))
        self.links = [(i, j, (ctypes.c_int * 6)(*box), (ctypes.c_int * 3)(*shift)) for i, j, box, shift in links]
        self.traces = None
        self.t = 0

    # -- ordering of the parts' streams ------------------------------------------
    def _parts_wait_main(self):
        for sub in self.subs:
            sub["stream"].wait_stream(self.stream)

    def _main_waits_parts(self):
        for sub in self.subs:
            self.stream.wait_stream(sub["stream"])

    def _barrier(self):
        """Everything enqueued so far on any part's stream comes before what
        any part enqueues next."""
        evs = []
        for sub in self.subs:
            e = torch.cuda.Event()
            e.record(sub["stream"])
            evs.append(e)
        for sub in self.subs:
            for e in evs:
                sub["stream"].wait_event(e)

    # -- set-up ----------------------------------------------------------------
    def _crop(self, vol, sub):
        (z0, z1), (y0, y1), (x0, x1) = sub["loc"]
        return vol[z0:z1, y0:y1, x0:x1].contiguous()

    def set_model(self, vel: torch.Tensor, rho: torch.Tensor | None = None):
        """The whole grid's model (and density), each part given its box.
        With 16-bit storage every part stores velocities at the whole model's
        maximum velocity (the scale one grid would use), so that exchanged
        values need no conversion."""
        self.c_max = float(vel.max())
        boxes = [(self._crop(vel, sub), None if rho is None else self._crop(rho, sub)) for sub in self.subs]
        self._parts_wait_main()   # the boxes are cut on the caller's stream
        for sub, (v, r) in zip(self.subs, boxes):
            sub["sim"].set_velocity_scale(self.c_max)
            sub["sim"].set_model(v, r)   # synchronises the part's stream

    def set_staggered(self, on: bool = True):
        for sub in self.subs:
            sub["sim"].set_staggered(on)

    def set_cpml_local(self, vel: torch.Tensor, R=1e-8, kappa_max=5.0, alpha_frac=0.05, q=3):
        """The local-velocity grading: every slab node's coefficients come
        from its own velocity and its face's layer, so each part computes
        them from its box of the model."""
        boxes = [self._crop(vel, sub) for sub in self.subs]
        self._parts_wait_main()
        for sub, v in zip(self.subs, boxes):
            sub["sim"].set_cpml_local(v, R=R, kappa_max=kappa_max, alpha_frac=alpha_frac, q=q)

    def set_cpml(self, R=1e-8, kappa_max=5.0, alpha_frac=0.05, q=3, c_ref=None):
        """The grading of the whole grid: one reference velocity (the whole
        model's maximum unless given) for every part."""
        c = float(c_ref) if c_ref else self.c_max
        for sub in self.subs:
            sub["sim"].set_cpml(R=R, kappa_max=kappa_max, alpha_frac=alpha_frac, q=q, c_ref=c)

    def inject(self, src_zyx, wavelet: torch.Tensor):
        """Every part whose box holds a shot's source injects it (the others
        get a zero wavelet row for that shot at a node of their own)."""
        src = [tuple(int(v) for v in r) for r in src_zyx]
        ws = []
        for sub in self.subs:
            loc = sub["loc"]
            rows, w = [], wavelet.clone()
            for k, node in enumerate(src):
                inside = all(loc[a][0] <= node[a] < loc[a][1] for a in range(3))
                if inside:
                    rows.append([node[a] - loc[a][0] for a in range(3)])
                else:
                    rows.append([0, 0, 0])
                    w[k].zero_()
            ws.append((sub, rows, w.contiguous()))
        self._parts_wait_main()
        for sub, rows, w in ws:
            sub["sim"].inject(rows, w)
        self._wavelets = ws   # kept alive until the parts have copied them

    def record(self, rec_zyx):
        """Receivers (global (z, y, x)); each is recorded by the part that
        owns it.  Returns the global traces tensor [nshots, nt_max, nrec]."""
        rec = [tuple(int(v) for v in r) for r in rec_zyx]
        self.traces = torch.zeros((self.nshots, self.nt_max, len(rec)), dtype=torch.float32, device=self.device)
        for sub in self.subs:
            own, loc = sub["own"], sub["loc"]
            cols = [i for i, r in enumerate(rec) if all(own[a][0] <= r[a] < own[a][1] for a in range(3))]
            sub["rec_cols"] = cols
            if cols:
                sub["sim"].record([[rec[i][a] - loc[a][0] for a in range(3)] for i in cols])
        return self.traces

    # -- stepping ----------------------------------------------------------------
    def exchange(self):
        for i, j, box, shift in self.links:
            a, b = self.subs[i]["sim"], self.subs[j]["sim"]
            a._check(a.lib.fdtd_exchange(a.ctx, b.ctx, box, shift))

    def step(self, n: int):
        """Advance n steps: blocks of s steps, each after a ghost exchange.
        The work is enqueued on the parts' streams, and the caller's stream
        waits for it before this returns."""
        self._parts_wait_main()
        done = 0
        while done < n:
            k = min(self.s, n - done)
            self._barrier()
            self.exchange()
            self._barrier()
            for sub in self.subs:
                sub["sim"].step(k)
            done += k
        self.t += n
        self._main_waits_parts()
        if self.traces is not None:
            for sub in self.subs:
                if sub["rec_cols"]:
                    self.traces[:, :, sub["rec_cols"]] = sub["sim"].traces

    def sync(self):
        for sub in self.subs:
            sub["sim"].sync()

    def reset(self):
        self._parts_wait_main()
        for sub in self.subs:
            sub["sim"].reset()
        self._main_waits_parts()
        self.t = 0

    def get(self, which: str, shot=0) -> torch.Tensor:
        """One field of the whole grid, assembled from the owned boxes."""
        out = torch.empty(self.shape, dtype=torch.float32, device=self.device)
        for sub in self.subs:
            loc, own = sub["loc"], sub["own"]
            # the part writes its field on its own stream into a buffer of the
            # caller's stream (which may reuse the previous part's buffer), so
            # it waits for the caller's stream first and the caller for it after
            sub["stream"].wait_stream(self.stream)
            f = sub["sim"].get(which, shot)
            self.stream.wait_stream(sub["stream"])
            sl = tuple(slice(o[0] - l[0], o[1] - l[0]) for o, l in zip(own, loc))
            out[own[0][0]:own[0][1], own[1][0]:own[1][1], own[2][0]:own[2][1]] = f[sl]
        return out

    def close(self):
        for sub in self.subs:
            sub["sim"].close()
        self.subs = []


__all__ = ["Decomposition", "plan", "split"]
