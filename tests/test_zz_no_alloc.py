"""The allocation-free sampling entry point (qs_sim_sample_noalloc).

It serves callers that cannot allocate device memory when they ask for
samples (a server that reserved the GPU up front for its own pool, a
framework whose allocator must own all device memory, a loop that cannot take
cudaFree's synchronisation): the frames live in a fixed static device array
inside libqs. This file is collected last on purpose, so that a run stopping
at the first failure has already run every other test; it also passes alone
in a fresh process, where the first call does the per-device set-up.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2603_14641_gb300 import qs  # noqa: E402
from workloads import circuits as C  # noqa: E402


def _noalloc(sim, shots, seed, on_device):
    M = sim.num_measurements
    ow = (shots + 63) // 64
    if on_device:
        out = torch.zeros((max(M, 1), ow), dtype=torch.int64, device=sim.device)
        qs.qs_sim_sample_noalloc(sim.sim, shots, seed, out.data_ptr(), M * ow)
        torch.cuda.synchronize()
        return out[:M].cpu().numpy().view(np.uint64)
    out = np.zeros((max(M, 1), ow), np.uint64)
    qs.qs_sim_sample_noalloc(sim.sim, shots, seed, out.ctypes.data, M * ow)
    return out[:M]


@pytest.mark.parametrize("device_resident", [False, True])
def test_noalloc_matches_sample_two_calls(device_resident):
    circ = C.gate_mix_circuit(300, 20, seed=12, measure_every=5, measure_frac=0.3)
    sim = qs.Simulator(circ.n, device="cuda:0")
    if device_resident:
        dc = sim.upload(circ)
        for op in circ.ops:
            if op[0] == "layers":
                sim.apply_layers_dev(dc, op[1], op[2])
            else:
                q = torch.from_numpy(np.asarray(op[1], np.uint32).view(np.int32)).cuda()
                sim.measure_dev(q, seed=3)
    else:
        sim.run(circ, seed=3)
    # two calls in a row, each checked against the workspace-based entry point
    for call, (shots, seed, on_dev) in enumerate([(1000, 77, True), (130, 78, False)]):
        want = sim.sample(shots, seed=seed, on_device=False)
        got = _noalloc(sim, shots, seed, on_dev)
        assert got.shape == want.shape
        assert np.array_equal(got, want), f"call {call} differs from qs_sim_sample"
    sim.sync()


def test_noalloc_rejects_oversize_request():
    sim = qs.Simulator(2000, device="cuda:0")
    sim.measure(np.arange(4, dtype=np.uint32), seed=1)
    shots = 64 * 2048  # 2 * 2000 * 2048 words = 62.5 MiB of frames > 32 MiB
    M, ow = 4, shots // 64
    out = torch.zeros((M, ow), dtype=torch.int64, device="cuda:0")
    with pytest.raises(qs.QsError) as e:
        qs.qs_sim_sample_noalloc(sim.sim, shots, 5, out.data_ptr(), M * ow)
    assert e.value.code == -5 and "static scratch" in str(e.value)
    sim.sync()  # nothing was enqueued; the sim is still usable


def test_noalloc_with_noise_channels_matches_sample():
    """The op log's noise channels (the replay_noise branch) go through the
    static array exactly as through a workspace."""
    circ = C.with_circuit_noise(C.gate_mix_circuit(120, 14, seed=5, measure_every=4,
                                                   measure_frac=0.3), 0.02, 0.05)
    sim = qs.Simulator(circ.n, device="cuda:0")
    sim.run(circ, seed=9)
    for shots, seed in [(700, 3), (64, 4)]:
        want = sim.sample(shots, seed=seed, on_device=False)
        assert np.array_equal(_noalloc(sim, shots, seed, True), want)
    sim.sync()


def test_noalloc_just_under_the_limit_and_allocates_nothing():
    """A request whose frames and record need just under QS_NOALLOC_SCRATCH_BYTES
    (n = 2000, 4 measurements, 66,816 shots: 2 * 2000 * 1044 * 8 + 4 * 1044 * 8
    = 33,441,408 of 33,554,432 bytes) succeeds and matches qs_sim_sample, and
    two calls in a row leave the device's free memory unchanged."""
    n, shots = 2000, 66_816
    circ = C.random_circuit(n, 6, 0.5, seed=3, final_measure_all=False)
    sim = qs.Simulator(n, device="cuda:0")
    sim.run(circ, seed=1)
    sim.measure(np.array([0, 1, 2, 3], np.uint32), seed=2)
    ow = (shots + 63) // 64
    fw = (ow + 3) // 4 * 4
    assert 2 * n * fw * 8 + 4 * ow * 8 <= (32 << 20) < 2 * n * (fw + 4) * 8 + 4 * (ow + 1) * 8
    want = sim.sample(shots, seed=11, on_device=True)
    out = torch.zeros((4, ow), dtype=torch.int64, device="cuda:0")
    qs.qs_sim_sample_noalloc(sim.sim, shots, 11, out.data_ptr(), 4 * ow)
    torch.cuda.synchronize()
    assert torch.equal(out, want)
    free1 = torch.cuda.mem_get_info()[0]
    qs.qs_sim_sample_noalloc(sim.sim, shots, 12, out.data_ptr(), 4 * ow)
    torch.cuda.synchronize()
    free2 = torch.cuda.mem_get_info()[0]
    assert free1 == free2, (free1, free2)
    assert torch.equal(out, sim.sample(shots, seed=12, on_device=True))
    sim.sync()
