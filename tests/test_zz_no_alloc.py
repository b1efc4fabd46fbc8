"""The allocation-free observe entry point gives the same counts as ka_observe.

Some callers cannot allocate device memory at all: an application whose
memory pool already owns the whole device heap, or a real-time loop where
cudaMalloc is forbidden.  ka_observe_static serves them: its per-replica
accumulators are a fixed array compiled into the library, and the caller
passes only the state (device, canonical layout) and a host output buffer.
This test calls it through the C ABI and checks that its counts equal those
of ka_observe, exactly (the counts are integers, so the tolerance is zero,
as in every parity test here), on two calls in a row.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU-only hosts
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1710_05155_gb300 as K  # noqa: E402


def test_static_observe_matches_ka_observe_twice():
    R = 256
    sim = K.Simulation(topo=K.KA_CUBIC, d=3, L=16, m=3, replicas=R)
    sim.init(3, 0.72)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        sim.sweep(7)
        sweep, want = sim.observe()
        assert sweep == 7 * (call + 1)
        n, n0, p = sim.get_state()
        dn, dn0, dp = (torch.from_numpy(x.view(np.int64)).cuda() for x in (n, n0, p))
        torch.cuda.synchronize()
        got = K.ka_observe_static(dn.data_ptr(), dn0.data_ptr(), dp.data_ptr(), sim.info["N"], R,
                                  stream)
        assert got.shape == (R, 4)
        assert (got == want).all(), f"call {call}: counts differ"
    sim.close()


def test_static_observe_rejects_too_many_replicas():
    x = torch.zeros((128, 16), dtype=torch.int64, device="cuda")
    with pytest.raises(K.KaError) as e:
        K.ka_observe_static(x.data_ptr(), x.data_ptr(), x.data_ptr(), 16, 8192)
    assert e.value.status == K.KA_EINVAL
