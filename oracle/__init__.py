"""Serial CPU oracle for the multispin Kob-Andersen chain (test infrastructure).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product library never imports, links or calls it, and it shares
no code with the CUDA path.

The arithmetic lives in ``ka_oracle.c`` (plain C, one byte per (site,
replica)); this module compiles it with gcc on first use and wraps it with
ctypes.  State arrays are numpy ``uint8`` of shape ``[N, Rs]`` (site-major).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ka_oracle.c")
_HDR = os.path.join(_HERE, "ka_oracle.h")
_SO = os.path.join(_HERE, "libka_oracle.so")
_lock = threading.Lock()
_lib = None

TAG_INIT = 0xFFFFFFFF
TAG_GRAPH = 0xFFFFFFFE


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (no GPU headers)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= newest:
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-Wall", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True, cwd=_HERE)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
        i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
        u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
        u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
        I64, U64, I = C.c_int64, C.c_uint64, C.c_int
        lib.ora_philox4x32_10.argtypes = [u32p, u32p, u32p]
        lib.ora_philox4x32_10.restype = None
        lib.ora_gate_word.argtypes = [U64, I64, I64, I64, I64]
        lib.ora_gate_word.restype = U64
        lib.ora_cubic_gate_word.argtypes = [U64, I64, I64, I64, I64, I]
        lib.ora_cubic_gate_word.restype = U64
        lib.ora_particles.argtypes = [C.c_double, I64]
        lib.ora_particles.restype = I64
        lib.ora_cubic_tables.argtypes = [I, I, i32p, i64p, i32p, i32p, i64p, C.POINTER(I64)]
        lib.ora_rrg_build.argtypes = [I64, I, U64, I64, i32p, C.POINTER(I64)]
        lib.ora_graph_edges.argtypes = [I64, I, i32p, i32p, i32p]
        lib.ora_graph_classes.argtypes = [I64, I, i32p, i64p, i32p, i32p, i64p, C.POINTER(I64)]
        lib.ora_check_schedule.argtypes = [I64, I, i32p, I64, i64p, i32p, i32p]
        lib.ora_local_move.argtypes = [I, I, I, I, u8p, u8p, I, C.POINTER(I), C.POINTER(I)]
        lib.ora_init.argtypes = [I64, I64, I64, U64, I64, u8p, u8p, u8p]
        lib.ora_class_step.argtypes = [I64, I, i32p, I, I64, i32p, i32p, i64p, I64, I64, U64,
                                       I64, I64, I, u8p, u8p]
        lib.ora_sweeps.argtypes = [I64, I, i32p, I, I64, i64p, i32p, i32p, i64p, U64, I64, I64,
                                   I, I64, I64, u8p, u8p]
        lib.ora_observe.argtypes = [I64, I64, u8p, u8p, u8p, i64p]
        lib.ora_observe.restype = None
        lib.ora_four_point.argtypes = [I, I, I64, u8p, u8p, I64, i64p, i64p]
        lib.ora_four_point.restype = I
        lib.ora_layered_graph.argtypes = [I, I, I, U64, i32p]
        lib.ora_layered_graph.restype = I
        lib.ora_sequential_sweeps.argtypes = [I64, I, i32p, I, U64, I64, I64, I64, I64, u8p, u8p]
        lib.ora_sequential_sweeps.restype = I
        for name in ("ora_cubic_tables", "ora_rrg_build", "ora_graph_edges", "ora_graph_classes",
                     "ora_check_schedule", "ora_local_move", "ora_init", "ora_class_step",
                     "ora_sweeps"):
            getattr(lib, name).restype = C.c_int
        _lib = lib
        return lib


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with status {rc}")


def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 block for a 4-word counter and a 2-word key."""
    out = np.zeros(4, np.uint32)
    _load().ora_philox4x32_10(np.asarray(ctr, np.uint32), np.asarray(key, np.uint32), out)
    return out


def gate_word(seed: int, t: int, cls: int, bond: int, w: int) -> int:
    """Gate word on a graph (edge id `bond`)."""
    return int(_load().ora_gate_word(seed, t, cls, bond, w))


def cubic_gate_word(seed: int, t: int, cls: int, bond: int, w: int, L: int) -> int:
    """Gate word on a periodic cubic lattice of side L (base site `bond`)."""
    return int(_load().ora_cubic_gate_word(seed, t, cls, bond, w, L))


def particles(rho: float, N: int) -> int:
    return int(_load().ora_particles(rho, N))


class Topology:
    """Neighbour table and bond classes of one lattice or graph."""

    def __init__(self, N, z, nbr, class_off, bu, bv, bid, cubic_L=0):
        self.N, self.z = int(N), int(z)
        self.cubic_L = int(cubic_L)  # side of a cubic lattice (its gate stream), 0 for graphs
        self.nbr = nbr
        self.class_off, self.bu, self.bv, self.bid = class_off, bu, bv, bid

    @property
    def nclass(self) -> int:
        return len(self.class_off) - 1

    def check(self) -> int:
        return int(_load().ora_check_schedule(self.N, self.z, self.nbr, self.nclass,
                                              self.class_off, self.bu, self.bv))


def cubic(d: int, L: int) -> Topology:
    lib = _load()
    N = L ** d
    z = 2 * d
    nc = 4 if d == 1 else 8 * d
    nbr = np.zeros(N * z, np.int32)
    off = np.zeros(nc + 1, np.int64)
    bu = np.zeros(d * N, np.int32)
    bv = np.zeros(d * N, np.int32)
    bid = np.zeros(d * N, np.int64)
    out = C.c_int64(0)
    _check(lib.ora_cubic_tables(d, L, nbr, off, bu, bv, bid, C.byref(out)), "cubic_tables")
    return Topology(N, z, nbr, off, bu, bv, bid, cubic_L=L)


def rrg_neighbours(N: int, z: int, graph_seed: int, max_attempts: int = 1 << 20):
    lib = _load()
    nbr = np.zeros(N * z, np.int32)
    att = C.c_int64(0)
    _check(lib.ora_rrg_build(N, z, graph_seed, max_attempts, nbr, C.byref(att)), "rrg_build")
    return nbr, int(att.value)


def graph_edges(N: int, z: int, nbr: np.ndarray):
    E = N * z // 2
    eu = np.zeros(E, np.int32)
    ev = np.zeros(E, np.int32)
    _check(_load().ora_graph_edges(N, z, np.ascontiguousarray(nbr, np.int32), eu, ev), "edges")
    return eu, ev


def graph(N: int, z: int, nbr: np.ndarray) -> Topology:
    lib = _load()
    nbr = np.ascontiguousarray(nbr, np.int32)
    E = N * z // 2
    off = np.zeros(E + 1, np.int64)
    bu = np.zeros(E, np.int32)
    bv = np.zeros(E, np.int32)
    bid = np.zeros(E, np.int64)
    nc = C.c_int64(0)
    _check(lib.ora_graph_classes(N, z, nbr, off, bu, bv, bid, C.byref(nc)), "graph_classes")
    return Topology(N, z, nbr, off[: nc.value + 1].copy(), bu, bv, bid)


def rrg(N: int, z: int, graph_seed: int) -> Topology:
    nbr, _ = rrg_neighbours(N, z, graph_seed)
    return graph(N, z, nbr)


def local_move(z: int, m: int, ni: int, nj: int, others_i, others_j, gate: int):
    a, b = C.c_int(0), C.c_int(0)
    _check(_load().ora_local_move(z, m, ni, nj, np.asarray(others_i, np.uint8),
                                  np.asarray(others_j, np.uint8), gate, C.byref(a), C.byref(b)),
           "local_move")
    return a.value, b.value


class State:
    """Occupation n, reference n0 and persistence p, bytes of shape [N, Rs]."""

    def __init__(self, N: int, Rs: int, r0: int = 0):
        self.N, self.Rs, self.r0 = int(N), int(Rs), int(r0)
        self.n = np.zeros((N, Rs), np.uint8)
        self.n0 = np.zeros((N, Rs), np.uint8)
        self.p = np.zeros((N, Rs), np.uint8)
        self.t = 0

    def copy(self) -> "State":
        s = State(self.N, self.Rs, self.r0)
        s.n, s.n0, s.p, s.t = self.n.copy(), self.n0.copy(), self.p.copy(), self.t
        return s


def init(N: int, R: int, seed: int, rho: float, r0: int = 0) -> State:
    st = State(N, R, r0)
    K = particles(rho, N)
    _check(_load().ora_init(N, r0, R, seed, K, st.n, st.n0, st.p), "init")
    return st


def class_step(topo: Topology, m: int, st: State, cls: int, seed: int, t: int | None = None):
    c0, c1 = int(topo.class_off[cls]), int(topo.class_off[cls + 1])
    _check(_load().ora_class_step(topo.N, topo.z, topo.nbr, m, c1 - c0,
                                  np.ascontiguousarray(topo.bu[c0:c1]),
                                  np.ascontiguousarray(topo.bv[c0:c1]),
                                  np.ascontiguousarray(topo.bid[c0:c1]),
                                  cls, st.t if t is None else t, seed, st.r0, st.Rs, topo.cubic_L,
                                  st.n, st.p),
           "class_step")


def sweeps(topo: Topology, m: int, st: State, seed: int, nsweeps: int) -> State:
    _check(_load().ora_sweeps(topo.N, topo.z, topo.nbr, m, topo.nclass, topo.class_off,
                              topo.bu, topo.bv, topo.bid, seed, st.r0, st.Rs, topo.cubic_L, st.t,
                              nsweeps, st.n, st.p), "sweeps")
    st.t += nsweeps
    return st


def observe(st: State) -> np.ndarray:
    """int64 [Rs, 4]: particles, overlap, persist_occ, persist_all."""
    out = np.zeros((st.Rs, 4), np.int64)
    _load().ora_observe(st.N, st.Rs, st.n, st.n0, st.p, out)
    return out


def four_point(d: int, L: int, st: State, smax: int):
    """(phi int64 [Rs, smax+1], psi int64 [smax+1]): ordered site pairs by shell
    s = |delta|^2 (components in [-L/2, L/2)), phi per replica of q_i q_j with
    q = n AND n0, psi of M_i M_j with M_i = sum over replicas of q_i."""
    phi = np.zeros((st.Rs, smax + 1), np.int64)
    psi = np.zeros(smax + 1, np.int64)
    _check(_load().ora_four_point(d, L, st.Rs, st.n, st.n0, smax, phi, psi), "four_point")
    return phi, psi


def sequential_sweeps(topo: Topology, m: int, st: State, seed: int, nsweeps: int) -> None:
    """Random-sequential sweeps (one random bond per attempt, shared by the 64
    replicas of a word; N attempts per sweep) from sweep st.t; advances st.t."""
    _check(_load().ora_sequential_sweeps(topo.N, topo.z, topo.nbr, m, seed, st.r0, st.Rs, st.t,
                                         nsweeps, st.n, st.p), "sequential_sweeps")
    st.t += nsweeps


def layered_graph(d: int, L: int, M: int, graph_seed: int) -> np.ndarray:
    """int32 [M L^d, 2d] neighbour rows of the layered random graph (section 5.2)."""
    N = L ** d
    nbr = np.zeros(M * N * 2 * d, np.int32)
    _check(_load().ora_layered_graph(d, L, M, graph_seed, nbr), "layered_graph")
    return nbr.reshape(M * N, 2 * d)


def pack_words(bits: np.ndarray) -> np.ndarray:
    """[N, R] bytes -> canonical [R/64, N] uint64 words (replica r = word r//64, bit r%64)."""
    N, R = bits.shape
    assert R % 64 == 0
    b = bits.reshape(N, R // 64, 64).astype(np.uint64)
    shifts = np.arange(64, dtype=np.uint64)
    words = (b << shifts).sum(axis=2, dtype=np.uint64)
    return np.ascontiguousarray(words.T)


def unpack_words(words: np.ndarray) -> np.ndarray:
    """canonical [W, N] uint64 words -> [N, 64*W] bytes."""
    W, N = words.shape
    shifts = np.arange(64, dtype=np.uint64)
    b = (words.T[:, :, None] >> shifts) & np.uint64(1)
    return np.ascontiguousarray(b.reshape(N, W * 64).astype(np.uint8))
