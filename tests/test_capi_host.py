"""Host-side checks of the C ABI library (no GPU needed).

The shared library must load and export every function include/ka.h
declares; parameter validation and the host topology builder run without a
device.  The library's lattices, random regular graphs and bond classes must
equal the oracle's (two independent implementations of one definition).
"""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle as O
import paper_1710_05155_gb300 as K

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?\w+\s*\**\s*(ka_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(K.load()._name)
    names = _declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    # the binding wraps exactly the declared functions
    assert sorted(K._SIGS) == names


def test_status_names():
    lib = K.load()
    assert lib.ka_status_name(0) == b"KA_OK"
    assert lib.ka_status_name(1) == b"KA_EINVAL"


@pytest.mark.parametrize("kw", [
    dict(topo=K.KA_CUBIC, d=3, L=18),          # L % 4 != 0
    dict(topo=K.KA_CUBIC, d=3, L=2),
    dict(topo=K.KA_CUBIC, d=5, L=8),
    dict(topo=K.KA_CUBIC, d=3, L=16, m=6),     # m > z - 1
    dict(topo=K.KA_CUBIC, d=3, L=16, m=-1),
    dict(topo=K.KA_CUBIC, d=3, L=16, replicas=100),
    dict(topo=K.KA_CUBIC, d=3, L=16, replicas=0),
    dict(topo=K.KA_RRG, N=7, z=3, m=2),         # N z odd
    dict(topo=K.KA_RRG, N=4, z=4, m=2),         # z >= N
    dict(topo=K.KA_RRG, N=100, z=9, m=2),       # z > 8
    dict(topo=K.KA_GRAPH, N=10, z=2, m=1),      # no neighbour list
    dict(topo=7, d=3, L=16),
])
def test_invalid_parameters_rejected(kw):
    p, _ = K.make_params(**kw)
    with pytest.raises(K.KaError) as e:
        K.ka_required_bytes(p)
    assert e.value.status == K.KA_EINVAL
    with pytest.raises(K.KaError) as e:
        K.ka_create(p)
    assert e.value.status == K.KA_EINVAL


def test_required_bytes_cover_the_planes():
    p, _ = K.make_params(topo=K.KA_CUBIC, d=3, L=128, m=3, replicas=256)
    nb = K.ka_required_bytes(p)
    plane = 128 ** 3 * 4 * 8
    assert 3 * plane <= nb < 4 * plane + (1 << 22)  # n, n0, p (+ a staging plane)
    p, _ = K.make_params(topo=K.KA_RRG, N=1 << 12, z=4, m=2, replicas=64)
    nb = K.ka_required_bytes(p)
    assert nb >= 3 * 4096 * 8 + 4096 * 4 * 4 + 3 * 8192 * 4


@pytest.mark.parametrize("d,L", [(1, 8), (2, 4), (2, 12), (3, 8), (4, 4)])
def test_cubic_tables_match_oracle(d, L):
    p, _ = K.make_params(topo=K.KA_CUBIC, d=d, L=L, m=0)
    t = K.ka_build_topology(p)
    o = O.cubic(d, L)
    z = 2 * d
    assert (t["class_off"] == o.class_off).all()
    assert (t["bu"] == o.bu).all() and (t["bv"] == o.bv).all() and (t["bid"] == o.bid).all()
    a = np.sort(t["nbr"].reshape(-1, z), axis=1)
    b = np.sort(o.nbr.reshape(-1, z), axis=1)
    assert (a == b).all()


@pytest.mark.parametrize("N,z,seed", [(64, 4, 1), (4096, 4, 1), (4096, 4, 7), (1000, 3, 2),
                                      (500, 6, 3), (33, 2, 5), (64, 5, 4),
                                      # large enough that attempts run on several threads
                                      (1 << 15, 4, 1), (30000, 3, 3)])
def test_rrg_matches_oracle(N, z, seed):
    p, _ = K.make_params(topo=K.KA_RRG, N=N, z=z, m=1, graph_seed=seed)
    t = K.ka_build_topology(p)
    o = O.rrg(N, z, seed)
    assert (t["nbr"] == o.nbr).all()
    assert (t["class_off"] == o.class_off).all()
    assert (t["bu"] == o.bu).all() and (t["bv"] == o.bv).all() and (t["bid"] == o.bid).all()


def test_caller_graph_matches_oracle_colouring():
    N, z = 300, 5
    nbr, _ = O.rrg_neighbours(N, z, 9)
    rows = nbr.reshape(N, z)[:, ::-1].copy()  # unsorted rows are accepted
    p, keep = K.make_params(topo=K.KA_GRAPH, N=N, z=z, m=2, nbr=rows)
    t = K.ka_build_topology(p)
    o = O.graph(N, z, nbr)
    assert (t["class_off"] == o.class_off).all()
    assert (t["bu"] == o.bu).all() and (t["bv"] == o.bv).all() and (t["bid"] == o.bid).all()


@pytest.mark.parametrize("bad", ["loop", "asym", "repeat", "range"])
def test_caller_graph_validation(bad):
    N, z = 20, 2
    ring = np.array([[(i - 1) % N, (i + 1) % N] for i in range(N)], np.int32)
    if bad == "loop":
        ring[3, 0] = 3
    elif bad == "asym":
        ring[3, 0] = 10
    elif bad == "repeat":
        ring[3] = [4, 4]
    else:
        ring[3, 1] = 99
    p, keep = K.make_params(topo=K.KA_GRAPH, N=N, z=z, m=1, nbr=ring)
    with pytest.raises(K.KaError):
        K.ka_build_topology(p)


@pytest.mark.parametrize("d,L,M,seed", [(3, 4, 2, 1), (3, 8, 16, 7), (2, 8, 8, 3), (1, 16, 3, 2),
                                        (4, 3, 2, 5), (3, 32, 4, 9)])  # the last one is threaded
def test_layered_graph_matches_oracle(d, L, M, seed):
    assert (K.ka_layered_graph(d, L, M, seed) == O.layered_graph(d, L, M, seed)).all()


@pytest.mark.parametrize("d,L,M", [(0, 4, 2), (5, 4, 2), (3, 2, 2), (3, 4, 0), (3, 4, 65536)])
def test_layered_graph_rejects(d, L, M):
    with pytest.raises(K.KaError) as e:
        K.ka_layered_graph(d, L, M, 1)
    assert e.value.status == K.KA_EINVAL


def test_asynchronous_state_load_checks_its_arrays():
    # rejected before the library is called: the copies read the caller's
    # memory after the call returns, so no temporary copy may stand in
    ctx = K.Ctx(0)
    ctx.info = {"words": 1, "N": 64}
    good = np.zeros((1, 64), np.uint64)
    for bad in (np.zeros((1, 128), np.uint64)[:, ::2], np.zeros((1, 64), np.int64), [0] * 64):
        with pytest.raises(ValueError):
            K.ka_set_state_async(ctx, bad, good, good, 0, 1)
    assert not ctx.inflight


@pytest.mark.parametrize("shape", [(1, 63), (2, 64), (0,), (1, 65)])
def test_state_load_checks_sizes(shape):
    # the library copies R/64 * N words from each host pointer: a shorter array
    # would be read past its end, a longer one silently truncated
    ctx = K.Ctx(0)
    ctx.info = {"words": 1, "N": 64}
    good = np.zeros((1, 64), np.uint64)
    bad = np.zeros(shape, np.uint64)
    for args in ((bad, good, good), (good, bad, good), (good, good, bad)):
        with pytest.raises(ValueError):
            K.ka_set_state_async(ctx, *args, 0, 1)
        with pytest.raises(ValueError):
            K.ka_set_state(ctx, *args, 0, 1)
    assert not ctx.inflight
