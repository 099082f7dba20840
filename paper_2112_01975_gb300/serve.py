"""Continuous-batching server for parameter-sweep solves.

Requests (a drop on D2Q9 or D3Q27 at some size, T/Tc and radius, a number
of steps, FP32 or FP16-shifted storage) arrive over time. The server keeps
every admitted lattice resident on the GPU, admits waiting requests in
arrival order as soon as their device-memory footprint fits the budget, and
advances all resident lattices of one lattice type and storage together with
one batched launch per step (lbm_batch_*), in ticks of a fixed number of
steps; a group's batch (its descriptors and captured graph) is kept from
tick to tick while its members do not change. A lattice that has finished
its steps is read back and freed at the end of its tick, which frees room
for the next arrivals. Every step of every solve runs in the library's
kernels; a member of a batch evolves bitwise as it would alone.

Latency runs from a request's arrival to its result on the host and
includes its host set-up: the EOS values (from a table built once when the
server starts, eos_tables.SetupTable) and the initial density field. The
host prepares arrived requests while the GPU runs a tick.

The one-at-a-time FP64 baseline solves the same requests in arrival order,
each alone on the GPU with FP64 storage, with the same set-up (the next
arrived request is prepared while the current one runs).
"""
from __future__ import annotations

import dataclasses
import hashlib
import math
import time

import numpy as np

from . import eos_tables, inputs
from .lbm import D2Q9, D3Q27, F16S, F32, F64, LBM, Batch, LBMError


@dataclasses.dataclass(frozen=True)
class Request:
    rid: int
    arrival: float        # seconds after the start of the sweep
    lattice: int          # 0 = D2Q9, 1 = D3Q27
    n: int                # side of the square/cubic periodic box
    t_over_tc: float
    radius_frac: float    # drop radius / n
    oscillating: bool     # n = 2 shape mode instead of a round drop
    steps: int
    seed: int
    storage: int = F32    # storage on the server (F32 or F16S)

    @property
    def nodes(self) -> int:
        return self.n ** (3 if self.lattice == D3Q27 else 2)


@dataclasses.dataclass
class Result:
    rid: int
    arrival: float
    done: float
    latency: float
    rho_min: float
    rho_max: float
    mass: float
    digest: str           # sha1 of the final populations ("" unless asked for)
    failed: bool = False  # a density became non-finite; the solve was dropped
    rho: np.ndarray | None = None   # the final density field, when kept


def sweep_requests(count: int = 512, rate: float = 50.0, seed: int = 5, steps: int = 5000,
                   sizes_2d=tuple(range(64, 513, 32)), sizes_3d=tuple(range(64, 193, 32)),
                   tr=(0.5, 0.95), radius=(0.15, 0.35), storages=(F32, F16S)) -> list[Request]:
    """Poisson arrivals (exponential gaps of mean 1/rate); each request a
    D2Q9 or D3Q27 drop with probability 1/2, size uniform over the given
    sides, T/Tc and radius fraction uniform in their ranges, round or n = 2
    oscillating with probability 1/2, storage uniform over the given ones.
    All draws from splitmix64(seed ^ k)."""
    u = (inputs.uniform_pm1(seed, 7 * count) + 1.0) / 2.0   # U[0, 1)
    u = u.reshape(count, 7)
    reqs, t = [], 0.0
    for k in range(count):
        t += -math.log(1.0 - u[k, 0]) / rate
        lat = D3Q27 if u[k, 1] >= 0.5 else D2Q9
        sizes = sizes_3d if lat == D3Q27 else sizes_2d
        n = sizes[min(int(u[k, 2] * len(sizes)), len(sizes) - 1)]
        reqs.append(Request(k, t, lat, n, tr[0] + (tr[1] - tr[0]) * u[k, 3],
                            radius[0] + (radius[1] - radius[0]) * u[k, 4], bool(u[k, 5] >= 0.5),
                            steps, 1000 + k,
                            storages[min(int(u[k, 6] * len(storages)), len(storages) - 1)]))
    return reqs


def setup(req: Request, width: float = 5.0, table=None):
    """EOS parameters and the initial density of a request (van der Waals,
    attraction scaled for a liquid dP/drho of 0.1, interface width 5); the
    lattice starts at rest in the physical velocity (lbm_init). table: an
    eos_tables.SetupTable of the EOS and width, else computed directly."""
    if table is not None:
        a, rv, rl, kappa = table(req.t_over_tc)
    else:
        a = eos_tables.stable_a(0, req.t_over_tc)
        rv, rl, _ = eos_tables.coexistence(0, req.t_over_tc, a)
        kappa = eos_tables.kappa_for_width(0, req.t_over_tc, a, width=width)
    tau = 0.8 if req.oscillating else 1.0
    n = req.n
    nz = n if req.lattice == D3Q27 else 1
    R0 = req.radius_frac * n
    if req.oscillating:
        # R(theta) = R0 (1 + eps cos 2 theta - eps^2 / 2), eps = 0.1 (Sec. 4.3 set-up)
        z, y, x = np.meshgrid(np.arange(nz), np.arange(n), np.arange(n), indexing="ij")
        dx, dy = x - n // 2, y - n // 2
        dz = (z - nz // 2) if nz > 1 else 0
        r = np.sqrt(dx ** 2 + dy ** 2 + dz ** 2)
        theta = np.arctan2(dy, dx)
        Rt = R0 * (1.0 + 0.1 * np.cos(2 * theta) - 0.005)
        rho = inputs.tanh_interface((r - Rt).ravel(), rl, rv, width)
    else:
        rho = inputs.drop(n, n, nz, R0, rv, rl, width=width)
    rho = inputs.add_noise(rho, 1e-4, req.seed)
    return dict(eos=0, t_over_tc=req.t_over_tc, kappa=kappa, tau=tau, a=a), rho


def footprint(req: Request, storage: int | None = None) -> int:
    nz = req.n if req.lattice == D3Q27 else 1
    return LBM.required_bytes(req.lattice, req.n, req.n, nz,
                              req.storage if storage is None else storage)


def _failed(req: Request, t0: float) -> Result:
    done = time.perf_counter() - t0
    return Result(req.rid, req.arrival, done, done - req.arrival, float("nan"), float("nan"),
                  float("nan"), "", failed=True)


def _finish(req: Request, g: LBM, t0: float, digest: bool = False, keep: bool = False) -> Result:
    rho = g.moments()[0]
    mass, _ = g.reduce()
    digest = hashlib.sha1(g.get_populations().tobytes()).hexdigest() if digest else ""
    done = time.perf_counter() - t0
    return Result(req.rid, req.arrival, done, done - req.arrival, float(rho.min()),
                  float(rho.max()), mass, digest, rho=rho if keep else None)


def _open(req: Request, storage: int, prepared) -> LBM:
    prm, rho = prepared[req.rid]
    nz = req.n if req.lattice == D3Q27 else 1
    g = LBM(req.lattice, req.n, req.n, nz, prm["eos"], prm["t_over_tc"], prm["kappa"],
            prm["tau"], a=prm["a"], storage=storage)
    g.init(rho)
    return g


class _Preparer:
    """Host set-up of requests that have arrived, once each, in arrival
    order; given set-ups (a dict rid -> setup) are used as they are."""

    def __init__(self, requests, table, given=None):
        self.order = sorted(requests, key=lambda r: r.arrival)
        self.table = table
        self.done = dict(given or {})
        self.k = 0

    def __getitem__(self, rid):
        return self.done[rid]

    def prepare(self, req):
        if req.rid not in self.done:
            self.done[req.rid] = setup(req, table=self.table)

    def prepare_arrived(self, now: float, realtime: bool, limit: int = 1 << 30):
        """Set up arrived requests not yet prepared (at most limit of them)."""
        while self.k < len(self.order) and limit > 0:
            req = self.order[self.k]
            if realtime and req.arrival > now:
                break
            if req.rid not in self.done:
                self.prepare(req)
                limit -= 1
            self.k += 1


def _table_for(requests, table):
    if table is not None:
        return table
    trs = [r.t_over_tc for r in requests]
    return eos_tables.SetupTable(0, min(trs), max(trs))


class Server:
    """Continuous batching with admission by device-memory footprint."""

    def __init__(self, hbm_budget: int, tick_steps: int = 50, digest: bool = False,
                 keep_fields: bool = False):
        self.hbm_budget = hbm_budget
        self.tick_steps = tick_steps
        self.digest = digest
        self.keep_fields = keep_fields
        self.batch_launches = 0
        self.batches_built = 0
        self.peak_resident = 0

    def run(self, requests, prepared=None, realtime: bool = True, table=None) -> list[Result]:
        """Serve the requests; prepared: set-ups computed beforehand (not
        counted in latency), else each request is set up after its arrival
        from table (an eos_tables.SetupTable; built here if None)."""
        prep = _Preparer(requests, None if prepared else _table_for(requests, table), prepared)
        pending = sorted(requests, key=lambda r: r.arrival)
        active = []            # [request, handle, steps left]
        groups = {}            # (lattice, storage) -> (member handles, Batch)
        used, results = 0, []
        t0 = time.perf_counter()
        while pending or active:
            now = time.perf_counter() - t0
            while pending and (pending[0].arrival <= now or not realtime):
                need = footprint(pending[0])
                if need > self.hbm_budget:
                    raise ValueError(f"request {pending[0].rid} needs {need} B > budget")
                if used + need > self.hbm_budget:
                    break
                req = pending.pop(0)
                prep.prepare(req)
                active.append([req, _open(req, req.storage, prep), req.steps])
                used += need
            self.peak_resident = max(self.peak_resident, len(active))
            if not active:
                if pending and realtime:
                    time.sleep(max(0.0, pending[0].arrival - (time.perf_counter() - t0)))
                continue
            k = min(self.tick_steps, min(a[2] for a in active))
            running = []
            for key in sorted({(a[0].lattice, a[0].storage) for a in active}):
                members = [a[1] for a in active if (a[0].lattice, a[0].storage) == key]
                old = groups.get(key)
                if old is None or old[0] != members:
                    if old is not None:
                        old[1].close()
                    groups[key] = (members, Batch(members))
                    self.batches_built += 1
                b = groups[key][1]
                l0 = b.launches
                b.step(k)              # the groups' launches overlap on the GPU
                running.append((key, b, l0))
            # host work while the GPU runs the tick: set up arrived requests
            prep.prepare_arrived(time.perf_counter() - t0, realtime)
            for key, b, l0 in running:
                try:
                    b.sync()
                except LBMError:
                    pass           # the members are checked one by one below
                self.batch_launches += b.launches - l0
            still, changed = [], set()
            for a in active:
                a[2] -= k
                try:
                    a[1].sync()
                    ok = True
                except LBMError:
                    ok = False     # isolate a diverged solve; the others go on
                if not ok or a[2] == 0:
                    key = (a[0].lattice, a[0].storage)
                    if key in groups and key not in changed:
                        groups.pop(key)[1].close()   # the members' buffers follow the batch
                        changed.add(key)
                    results.append(_finish(a[0], a[1], t0, self.digest, self.keep_fields)
                                   if ok else _failed(a[0], t0))
                    a[1].close()
                    used -= footprint(a[0])
                else:
                    still.append(a)
            active = still
        for members, b in groups.values():
            b.close()
        return results


def run_sequential_f64(requests, prepared=None, realtime: bool = True, table=None,
                       keep_fields: bool = False) -> list[Result]:
    """One request at a time, FP64 storage, in arrival order; the next
    arrived request is set up while the current one runs."""
    prep = _Preparer(requests, None if prepared else _table_for(requests, table), prepared)
    results = []
    t0 = time.perf_counter()
    for req in sorted(requests, key=lambda r: r.arrival):
        if realtime:
            time.sleep(max(0.0, req.arrival - (time.perf_counter() - t0)))
        prep.prepare(req)
        g = _open(req, F64, prep)
        g.step(req.steps)
        prep.prepare_arrived(time.perf_counter() - t0, realtime, limit=1)
        try:
            g.sync()
            results.append(_finish(req, g, t0, keep=keep_fields))
        except LBMError:
            results.append(_failed(req, t0))
        g.close()
    return results


def summarize(results) -> dict:
    ok = [r for r in results if not r.failed]
    lat = np.array([r.latency for r in ok])
    span = max(r.done for r in results) - min(r.arrival for r in results)
    return {"solves": len(ok), "failed": len(results) - len(ok), "solves_per_s": len(ok) / span,
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "makespan_s": span}
