"""Python binding of the GB300 multispin Kob-Andersen library (include/ka.h).

A thin ctypes layer over the C ABI: the functions keep the C names and only
marshal arguments.  Every step of the dynamics runs in the CUDA library; if
the library cannot be loaded, the calls raise instead of falling back to
anything else.  PyTorch supplies device memory (``Simulation`` allocates the
context buffer as a torch tensor) and the CUDA stream.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

KA_OK, KA_EINVAL, KA_ENOMEM, KA_ECUDA, KA_ETIMEOUT, KA_EBUSY, KA_ESTATE = range(7)
KA_CUBIC, KA_RRG, KA_GRAPH = 0, 1, 2
KA_FLAG_GENERIC = 1

_STATUS = {0: "KA_OK", 1: "KA_EINVAL", 2: "KA_ENOMEM", 3: "KA_ECUDA", 4: "KA_ETIMEOUT",
           5: "KA_EBUSY", 6: "KA_ESTATE"}


class KaError(RuntimeError):
    def __init__(self, status: int, where: str, message: str = ""):
        self.status = status
        super().__init__(f"{where}: {_STATUS.get(status, status)}" + (f" ({message})" if message else ""))


class ka_params(C.Structure):
    _fields_ = [("topo", C.c_int32), ("d", C.c_int32), ("L", C.c_int32), ("z", C.c_int32),
                ("N", C.c_int64), ("m", C.c_int32), ("replicas", C.c_int32),
                ("graph_seed", C.c_uint64), ("nbr", C.POINTER(C.c_int32)),
                ("stream", C.c_void_p), ("device", C.c_int32), ("flags", C.c_int32)]


class ka_job_spec(C.Structure):
    _fields_ = [("sweeps", C.c_int64), ("observe_every", C.c_int64), ("seed", C.c_uint64),
                ("rho", C.c_double)]


KA_BATCH_GRAPH, KA_BATCH_PLAIN = 1, 2


class ka_info_t(C.Structure):
    _fields_ = [("N", C.c_int64), ("z", C.c_int32), ("m", C.c_int32), ("replicas", C.c_int32),
                ("words", C.c_int32), ("nclass", C.c_int64), ("nbonds", C.c_int64),
                ("sweep", C.c_int64), ("K", C.c_int64), ("seed", C.c_uint64),
                ("kernel", C.c_int32), ("rrg_attempts", C.c_int32), ("device_bytes", C.c_size_t),
                ("planes", C.c_int32), ("plane_words", C.c_int32),
                ("planes_per_launch", C.c_int32)]


_lib = None

# every symbol include/ka.h declares, with (restype, argtypes)
_P = C.POINTER
_SIGS = {
    "ka_required_bytes": (C.c_int, [_P(ka_params), _P(C.c_size_t)]),
    "ka_create": (C.c_int, [_P(ka_params), _P(C.c_void_p)]),
    "ka_create_in": (C.c_int, [_P(ka_params), C.c_void_p, C.c_size_t, _P(C.c_void_p)]),
    "ka_init": (C.c_int, [C.c_void_p, C.c_uint64, C.c_double]),
    "ka_sweep": (C.c_int, [C.c_void_p, C.c_int64]),
    "ka_observe": (C.c_int, [C.c_void_p, _P(C.c_int64), C.c_void_p]),
    "ka_observe_device": (C.c_int, [C.c_void_p, C.c_void_p]),
    "ka_get_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ka_set_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                               C.c_uint64]),
    "ka_set_state_async": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                                     C.c_uint64]),
    "ka_sync": (C.c_int, [C.c_void_p]),
    "ka_info": (C.c_int, [C.c_void_p, _P(ka_info_t)]),
    "ka_graph_tables": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_void_p]),
    "ka_build_topology": (C.c_int, [_P(ka_params), _P(C.c_int64), _P(C.c_int64), C.c_void_p,
                              C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ka_profile_enable": (C.c_int, [C.c_void_p, C.c_int32]),
    "ka_profile_read": (C.c_int, [C.c_void_p, _P(C.c_double), _P(C.c_int64)]),
    "ka_profile_read_dirs": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "ka_observe_static": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int32,
                                    C.c_void_p, C.c_void_p]),
    "ka_batch_create": (C.c_int, [C.c_int32, C.c_void_p, C.c_size_t, C.c_int32, _P(C.c_void_p)]),
    "ka_batch_add": (C.c_int, [C.c_void_p, _P(ka_params), _P(ka_job_spec), _P(C.c_int64)]),
    "ka_job_bytes": (C.c_int, [_P(ka_params), _P(ka_job_spec), _P(C.c_size_t)]),
    "ka_four_point": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]),
    "ka_layered_graph": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.c_uint64, C.c_void_p]),
    "ka_sweep_sequential": (C.c_int, [C.c_void_p, C.c_int64]),
    "ka_batch_adopt": (C.c_int, [C.c_void_p, C.c_void_p, _P(ka_job_spec), _P(C.c_int64)]),
    "ka_batch_step": (C.c_int, [C.c_void_p, C.c_int64, _P(C.c_int64)]),
    "ka_batch_autotune": (C.c_int, [C.c_void_p, _P(C.c_int64)]),
    "ka_batch_poll": (C.c_int, [C.c_void_p, C.c_int64, _P(C.c_int64), _P(C.c_int32)]),
    "ka_batch_state": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ka_batch_tuning": (C.c_int, [C.c_void_p, _P(C.c_int64), _P(C.c_int64)]),
    "ka_batch_observations": (C.c_int, [C.c_void_p, C.c_int64, _P(C.c_int64), C.c_void_p,
                                        C.c_void_p]),
    "ka_batch_remove": (C.c_int, [C.c_void_p, C.c_int64]),
    "ka_batch_info": (C.c_int, [C.c_void_p, _P(C.c_size_t), _P(C.c_int64), _P(C.c_int64)]),
    "ka_batch_destroy": (C.c_int, [C.c_void_p]),
    "ka_destroy": (C.c_int, [C.c_void_p]),
    "ka_last_error": (C.c_char_p, [C.c_void_p]),
    "ka_status_name": (C.c_char_p, [C.c_int]),
}


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load the CUDA library (building it with nvcc if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"CUDA library not built: {_build.LIB}")
    lib = C.CDLL(_build.LIB)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _ptr(a) -> C.c_void_p:
    return C.c_void_p(a.ctypes.data) if a is not None else C.c_void_p(0)


class Ctx:
    """An opaque ka_ctx* plus the objects that must outlive it."""

    def __init__(self, handle: int, keep=()):
        self.handle = C.c_void_p(handle)
        self._keep = keep  # any objects the context must not outlive
        self.info = None
        self.inflight = []  # host arrays of queued copies, until the next synchronisation

    def __bool__(self):
        return bool(self.handle.value)


def _check(status: int, where: str, ctx: Ctx | None = None) -> None:
    if status != KA_OK:
        msg = ""
        if ctx is not None and ctx.handle.value:
            msg = load().ka_last_error(ctx.handle).decode()
        raise KaError(status, where, msg)


def make_params(topo: int = KA_CUBIC, d: int = 3, L: int = 16, z: int = 0, N: int = 0, m: int = 3,
                replicas: int = 64, graph_seed: int = 1, nbr=None, stream: int | None = None,
                device: int = 0, flags: int = 0):
    p = ka_params()
    p.topo, p.d, p.L, p.z, p.N, p.m = topo, d, L, z, N, m
    p.replicas, p.graph_seed, p.device, p.flags = replicas, graph_seed, device, flags
    keep = None
    if nbr is not None:
        keep = np.ascontiguousarray(nbr, np.int32)
        p.nbr = keep.ctypes.data_as(C.POINTER(C.c_int32))
    p.stream = stream or 0
    return p, keep


def ka_required_bytes(params: ka_params) -> int:
    out = C.c_size_t(0)
    _check(load().ka_required_bytes(C.byref(params), C.byref(out)), "ka_required_bytes")
    return out.value


def ka_job_bytes(params: ka_params, sweeps: int, observe_every: int) -> int:
    """Device bytes a job takes from a batch's budget (context + observations)."""
    out = C.c_size_t(0)
    spec = ka_job_spec(sweeps, observe_every, 0, 0.0)
    _check(load().ka_job_bytes(C.byref(params), C.byref(spec), C.byref(out)), "ka_job_bytes")
    return out.value


def ka_layered_graph(d: int, L: int, M: int, graph_seed: int) -> np.ndarray:
    """int32 [M L^d, 2d] neighbour rows of the layered random graph (section 5.2):
    pass them as KA_GRAPH with N = M L^d, z = 2d."""
    nbr = np.zeros((M * L ** d, 2 * d), np.int32)
    _check(load().ka_layered_graph(d, L, M, graph_seed, _ptr(nbr)), "ka_layered_graph")
    return nbr


def ka_create(params: ka_params, keep=()) -> Ctx:
    h = C.c_void_p(0)
    _check(load().ka_create(C.byref(params), C.byref(h)), "ka_create")
    ctx = Ctx(h.value, keep)
    ctx.info = ka_info(ctx)
    return ctx


def ka_create_in(params: ka_params, device_ptr: int, nbytes: int, keep=()) -> Ctx:
    h = C.c_void_p(0)
    _check(load().ka_create_in(C.byref(params), C.c_void_p(device_ptr), nbytes, C.byref(h)),
           "ka_create_in")
    ctx = Ctx(h.value, keep)
    ctx.info = ka_info(ctx)
    return ctx


def ka_init(ctx: Ctx, seed: int, rho: float) -> None:
    _check(load().ka_init(ctx.handle, seed, rho), "ka_init", ctx)


def ka_sweep(ctx: Ctx, n: int) -> None:
    _check(load().ka_sweep(ctx.handle, n), "ka_sweep", ctx)


def ka_sweep_sequential(ctx: Ctx, n: int) -> None:
    """n sweeps of the random-sequential schedule (one bond per attempt, shared by the
    replicas of a word; N attempts per sweep)."""
    _check(load().ka_sweep_sequential(ctx.handle, n), "ka_sweep_sequential", ctx)


def ka_info(ctx: Ctx) -> dict:
    info = ka_info_t()
    _check(load().ka_info(ctx.handle, C.byref(info)), "ka_info", ctx)
    return {k: getattr(info, k) for k, _ in ka_info_t._fields_}


def ka_observe(ctx: Ctx, out: np.ndarray | None = None):
    """(sweep, int64 [R, 4]): particles, overlap, persist_occ, persist_all per replica."""
    R = ka_info(ctx)["replicas"]
    if out is None:
        out = np.zeros((R, 4), np.int64)
    sweep = C.c_int64(0)
    _check(load().ka_observe(ctx.handle, C.byref(sweep), _ptr(out)), "ka_observe", ctx)
    ctx.inflight.clear()
    return sweep.value, out


def ka_four_point(ctx: Ctx, smax: int, with_psi: bool = True):
    """(phi int64 [R, smax+1], psi int64 [smax+1] or None): four-point sums by shell
    s = |delta|^2 (section 2.2 g_4, section 3.3 Phi); see include/ka.h."""
    R = ka_info(ctx)["replicas"]
    phi = np.zeros((R, smax + 1), np.int64)
    psi = np.zeros(smax + 1, np.int64) if with_psi else None
    _check(load().ka_four_point(ctx.handle, smax, _ptr(phi), _ptr(psi) if with_psi else None),
           "ka_four_point", ctx)
    return phi, psi


def ka_observe_device(ctx: Ctx, counts_device_ptr: int) -> None:
    _check(load().ka_observe_device(ctx.handle, C.c_void_p(counts_device_ptr)),
           "ka_observe_device", ctx)


def ka_get_state(ctx: Ctx):
    """Host copies (n, n0, p), each uint64 [R/64, N] in canonical layout."""
    info = ka_info(ctx)
    shape = (info["words"], info["N"])
    n, n0, p = (np.zeros(shape, np.uint64) for _ in range(3))
    _check(load().ka_get_state(ctx.handle, _ptr(n), _ptr(n0), _ptr(p)), "ka_get_state", ctx)
    ctx.inflight.clear()
    return n, n0, p


def _check_state_sizes(ctx: Ctx, arrays, where: str) -> None:
    """Each state array must hold exactly R/64 * N words: the library copies
    that many from every host pointer."""
    info = ctx.info if ctx.info is not None else ka_info(ctx)
    need = int(info["words"]) * int(info["N"])
    for x in arrays:
        if x.size != need:
            raise ValueError(f"{where}: every array must hold R/64 * N = {need} words "
                             f"(shape (R/64, N)), got {x.size}")


def ka_set_state(ctx: Ctx, n, n0, p, sweep: int, seed: int) -> None:
    n, n0, p = (np.ascontiguousarray(x, np.uint64) for x in (n, n0, p))
    _check_state_sizes(ctx, (n, n0, p), "ka_set_state")
    _check(load().ka_set_state(ctx.handle, _ptr(n), _ptr(n0), _ptr(p), sweep, seed),
           "ka_set_state", ctx)
    ctx.inflight.clear()


def ka_set_state_async(ctx: Ctx, n, n0, p, sweep: int, seed: int) -> None:
    """ka_set_state queued on the context's stream without synchronising.  n, n0
    and p must be C-contiguous uint64 arrays (page-locked for the copies to be
    asynchronous); they are kept referenced until the next ka_sync of ctx and
    must not be changed before it."""
    for x in (n, n0, p):
        if not (isinstance(x, np.ndarray) and x.dtype == np.uint64 and x.flags.c_contiguous):
            raise ValueError("ka_set_state_async needs C-contiguous uint64 arrays")
    _check_state_sizes(ctx, (n, n0, p), "ka_set_state_async")
    _check(load().ka_set_state_async(ctx.handle, _ptr(n), _ptr(n0), _ptr(p), sweep, seed),
           "ka_set_state_async", ctx)
    ctx.inflight.append((n, n0, p))


def ka_sync(ctx: Ctx) -> None:
    _check(load().ka_sync(ctx.handle), "ka_sync", ctx)
    ctx.inflight.clear()


def ka_graph_tables(ctx: Ctx) -> dict:
    info = ka_info(ctx)
    N, z, E, C_ = info["N"], info["z"], info["nbonds"], info["nclass"]
    t = {"nbr": np.zeros(N * z, np.int32), "class_off": np.zeros(C_ + 1, np.int64),
         "bu": np.zeros(E, np.int32), "bv": np.zeros(E, np.int32), "bid": np.zeros(E, np.int64)}
    _check(load().ka_graph_tables(ctx.handle, _ptr(t["nbr"]), _ptr(t["class_off"]), _ptr(t["bu"]),
                                  _ptr(t["bv"]), _ptr(t["bid"])), "ka_graph_tables", ctx)
    return t


def ka_build_topology(params: ka_params) -> dict:
    """Host-only topology tables (no device): nbr, class_off, bu, bv, bid."""
    lib = load()
    nc, nb = C.c_int64(0), C.c_int64(0)
    _check(lib.ka_build_topology(C.byref(params), C.byref(nc), C.byref(nb), None, None, None, None,
                           None), "ka_build_topology")
    N = params.N if params.topo != KA_CUBIC else params.L ** params.d
    z = params.z if params.topo != KA_CUBIC else 2 * params.d
    t = {"nbr": np.zeros(N * z, np.int32), "class_off": np.zeros(nb.value + 1, np.int64),
         "bu": np.zeros(nb.value, np.int32), "bv": np.zeros(nb.value, np.int32),
         "bid": np.zeros(nb.value, np.int64)}
    _check(lib.ka_build_topology(C.byref(params), C.byref(nc), C.byref(nb), _ptr(t["nbr"]),
                           _ptr(t["class_off"]), _ptr(t["bu"]), _ptr(t["bv"]), _ptr(t["bid"])),
           "ka_build_topology")
    t["class_off"] = t["class_off"][: nc.value + 1].copy()
    return t


def ka_profile_enable(ctx: Ctx, enable: bool) -> None:
    _check(load().ka_profile_enable(ctx.handle, 1 if enable else 0), "ka_profile_enable", ctx)


def ka_profile_read(ctx: Ctx):
    ms, n = C.c_double(0), C.c_int64(0)
    _check(load().ka_profile_read(ctx.handle, C.byref(ms), C.byref(n)), "ka_profile_read", ctx)
    return ms.value, n.value


def ka_profile_read_dirs(ctx: Ctx):
    """Summed kernel ms [4] and launches [4] by bond direction since the last read."""
    ms, n = np.zeros(4, np.float64), np.zeros(4, np.int64)
    _check(load().ka_profile_read_dirs(ctx.handle, _ptr(ms), _ptr(n)), "ka_profile_read_dirs", ctx)
    return ms, n


def ka_observe_static(n_ptr: int, n0_ptr: int, p_ptr: int, N: int, replicas: int,
                      stream: int | None = None) -> np.ndarray:
    """Counts [R, 4] of caller-held device state (canonical [R/64, N] layout),
    computed without allocating: the accumulators are a fixed array inside the
    library (at most 4096 replicas)."""
    out = np.zeros((replicas, 4), np.int64)
    _check(load().ka_observe_static(C.c_void_p(n_ptr), C.c_void_p(n0_ptr), C.c_void_p(p_ptr), N,
                                    replicas, _ptr(out), C.c_void_p(stream or 0)),
           "ka_observe_static")
    return out


def ka_destroy(ctx: Ctx) -> None:
    if ctx and ctx.handle.value:
        st = load().ka_destroy(ctx.handle)
        ctx.handle = C.c_void_p(0)
        _check(st, "ka_destroy")


def ka_last_error(ctx: Ctx) -> str:
    return load().ka_last_error(ctx.handle).decode()


class Batch:
    """Many independent jobs resident on one device, advanced together (batch API)."""

    def __init__(self, device: int = 0, stream: int | None = None, hbm_budget: int = 150 << 30,
                 flags: int = KA_BATCH_GRAPH):
        h = C.c_void_p(0)
        _check(load().ka_batch_create(device, C.c_void_p(stream or 0), hbm_budget, flags,
                                      C.byref(h)), "ka_batch_create")
        self.handle = h
        self.device = device

    def add(self, sweeps: int, observe_every: int, seed: int, rho: float, **params) -> int:
        """Admit a job; returns its id.  Raises KaError(KA_EBUSY) when over budget."""
        p, keep = make_params(device=self.device, **params)
        spec = ka_job_spec(sweeps, observe_every, seed, rho)
        jid = C.c_int64(0)
        _check(load().ka_batch_add(self.handle, C.byref(p), C.byref(spec), C.byref(jid)),
               "ka_batch_add")
        return jid.value

    def adopt(self, ctx: Ctx, sweeps: int, observe_every: int) -> int:
        """Admit an initialised context made by ka_create; the batch takes it over.

        Raises KaError(KA_EBUSY) when over budget (the context stays the caller's)."""
        spec = ka_job_spec(sweeps, observe_every, 0, 0.0)
        jid = C.c_int64(0)
        _check(load().ka_batch_adopt(self.handle, ctx.handle, C.byref(spec), C.byref(jid)),
               "ka_batch_adopt")
        ctx.handle = C.c_void_p(0)
        return jid.value

    def step(self, max_sweeps: int = 0) -> int:
        ran = C.c_int64(0)
        _check(load().ka_batch_step(self.handle, max_sweeps, C.byref(ran)), "ka_batch_step")
        return ran.value

    def autotune(self) -> int:
        k = C.c_int64(0)
        _check(load().ka_batch_autotune(self.handle, C.byref(k)), "ka_batch_autotune")
        return k.value

    def tuning(self):
        """(round length, own-launch tile threshold) the batch uses now."""
        k, t = C.c_int64(0), C.c_int64(0)
        _check(load().ka_batch_tuning(self.handle, C.byref(k), C.byref(t)), "ka_batch_tuning")
        return k.value, t.value

    def poll(self, job: int):
        t, f = C.c_int64(0), C.c_int32(0)
        _check(load().ka_batch_poll(self.handle, job, C.byref(t), C.byref(f)), "ka_batch_poll")
        return t.value, bool(f.value)

    def observations(self, job: int, replicas: int):
        """(sweeps [n_obs], counts [n_obs, R, 4]) of a job."""
        n = C.c_int64(0)
        _check(load().ka_batch_observations(self.handle, job, C.byref(n), None, None),
               "ka_batch_observations")
        sw = np.zeros(n.value, np.int64)
        cnt = np.zeros((n.value, replicas, 4), np.int64)
        _check(load().ka_batch_observations(self.handle, job, C.byref(n), _ptr(sw), _ptr(cnt)),
               "ka_batch_observations")
        return sw, cnt

    def state(self, job: int, words: int, N: int):
        """(n, n0, p) of a job, each [R/64, N] uint64 in canonical layout."""
        out = [np.zeros((words, N), np.uint64) for _ in range(3)]
        _check(load().ka_batch_state(self.handle, job, *(_ptr(a) for a in out)), "ka_batch_state")
        return tuple(out)

    def remove(self, job: int) -> None:
        _check(load().ka_batch_remove(self.handle, job), "ka_batch_remove")

    def info(self):
        used, jobs, active = C.c_size_t(0), C.c_int64(0), C.c_int64(0)
        _check(load().ka_batch_info(self.handle, C.byref(used), C.byref(jobs), C.byref(active)),
               "ka_batch_info")
        return {"used_bytes": used.value, "jobs": jobs.value, "active": active.value}

    def close(self) -> None:
        if self.handle.value:
            st = load().ka_batch_destroy(self.handle)
            self.handle = C.c_void_p(0)
            _check(st, "ka_batch_destroy")

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Simulation:
    """One context whose device buffer is a torch tensor on torch's current stream.

    >>> sim = Simulation(topo=KA_CUBIC, d=3, L=16, m=3, replicas=64)
    >>> sim.init(seed=1, rho=0.7); sim.sweep(10); sweep, counts = sim.observe()
    """

    def __init__(self, device: int = 0, stream=None, **kw):
        import torch

        self.device = device
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        params, keep = make_params(stream=stream.cuda_stream, device=device, **kw)
        nbytes = ka_required_bytes(params)
        self.buffer = torch.empty(nbytes, dtype=torch.uint8, device=f"cuda:{device}")
        self.ctx = ka_create_in(params, self.buffer.data_ptr(), nbytes, keep=(keep, self.buffer))
        self.info = ka_info(self.ctx)

    def init(self, seed: int, rho: float) -> None:
        ka_init(self.ctx, seed, rho)

    def sweep(self, n: int) -> None:
        ka_sweep(self.ctx, n)

    def sweep_sequential(self, n: int) -> None:
        ka_sweep_sequential(self.ctx, n)

    def observe(self):
        return ka_observe(self.ctx)

    def get_state(self):
        return ka_get_state(self.ctx)

    def four_point(self, smax: int, with_psi: bool = True):
        return ka_four_point(self.ctx, smax, with_psi)

    def set_state(self, n, n0, p, sweep: int, seed: int) -> None:
        ka_set_state(self.ctx, n, n0, p, sweep, seed)

    def set_state_async(self, n, n0, p, sweep: int, seed: int) -> None:
        ka_set_state_async(self.ctx, n, n0, p, sweep, seed)

    def close(self) -> None:
        ka_destroy(self.ctx)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            if self.ctx:
                ka_destroy(self.ctx)
        except Exception:
            pass


def correlation(counts: np.ndarray, N: int, K: int) -> float:
    """C(t) of section 3.3 averaged over replicas, rho = K / N."""
    rho = K / N
    return float(((counts[:, 1] - N * rho * rho) / (N * rho * (1.0 - rho))).mean())


def persistence(counts: np.ndarray, K: int) -> float:
    """Fraction of the initial particles whose site has never changed."""
    return float((counts[:, 2] / K).mean())


def susceptibility(counts: np.ndarray, N: int, K: int) -> float:
    """Dynamical susceptibility chi_4(t) of section 2.2: N times the variance, over
    replicas (the average over initial configurations), of the overlap
    q_r(t) = (sum_i n_i(t) n_i(0) - N rho^2) / (N rho (1 - rho)), rho = K / N.

    counts: int64 [R, 4] as returned by ka_observe.  Replica averages are plain
    means over the R replicas.  chi_4(0) = 0; for independent uniform
    configurations (the ergodic long-time limit) its expectation is N / (N - 1).
    """
    rho = K / N
    q = (counts[:, 1] - N * rho * rho) / (N * rho * (1.0 - rho))
    return float(N * (np.mean(q * q) - np.mean(q) ** 2))


def four_point_g4(phi: np.ndarray, psi: np.ndarray, N: int, K: int) -> np.ndarray:
    """g_4(r, t) of section 2.2 per shell s = r^2, from ka_four_point's outputs.

    g4[s] = sum over ordered pairs (i, j) in shell s of (<q_i q_j> - <q_i><q_j>),
    divided by N rho^2 (1 - rho)^2, with <.> the mean over the R replicas:
    <q_i q_j> summed over the shell is phi[:, s].sum() / R and <q_i><q_j> is
    psi[s] / R^2.  Summed over every shell of the lattice it equals chi_4(t).
    """
    R = phi.shape[0]
    rho = K / N
    return (phi.sum(axis=0) / R - psi / (R * R)) / (N * rho * rho * (1.0 - rho) ** 2)
