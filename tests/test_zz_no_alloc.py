"""The allocation-free energy entry point (gsb_energy_noalloc), for callers
that cannot call cudaMalloc: it must give the same energies as gsb_energy on
consecutive calls that share its fixed scratch array. Collected last on
purpose, so a failure here comes after every other test has run."""
import numpy as np
import pytest

from paper_2508_17655_gb300 import gsb, inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2508_17655_gb300 import build
    build.build()


def _spins(R, N, seed):
    return (np.random.default_rng(seed).integers(0, 2, size=(R, N)) * 2 - 1).astype(np.int8)


@pytest.mark.parametrize("kind", ["pm1", "gauss"])
def test_noalloc_energy_matches_gsb_energy_on_two_calls(kind):
    torch = pytest.importorskip("torch")
    N, R = 300, 203
    J = I.sk_pm1(N, 3).astype(np.float32) if kind == "pm1" else I.sk_gauss(N, 3)
    P = gsb.Problem.dense(J)
    Jd = torch.from_numpy(np.ascontiguousarray(J)).cuda()
    stream = torch.cuda.current_stream()
    for call, seed in enumerate((11, 12)):  # two calls in a row, different spins
        S = _spins(R, N, seed)
        ref = P.energy(S)
        Sd = torch.from_numpy(S).cuda()
        Ed = torch.full((R,), float("nan"), dtype=torch.float64, device="cuda")
        gsb.energy_noalloc(Jd.data_ptr(), N, Sd.data_ptr(), R, Ed.data_ptr(), stream=stream)
        torch.cuda.synchronize()
        got = Ed.cpu().numpy()
        if kind == "pm1":
            np.testing.assert_array_equal(got, ref)  # integer J: exact on both sides
        else:
            np.testing.assert_allclose(got, ref, rtol=1e-5, atol=1e-5)


def test_noalloc_rejects_more_replicas_than_its_scratch():
    torch = pytest.importorskip("torch")
    N, R = 4, 65537
    Jd = torch.zeros((N, N), dtype=torch.float32, device="cuda")
    Sd = torch.ones((R, N), dtype=torch.int8, device="cuda")
    Ed = torch.zeros((R,), dtype=torch.float64, device="cuda")
    with pytest.raises(gsb.GsbError) as e:
        gsb.energy_noalloc(Jd.data_ptr(), N, Sd.data_ptr(), R, Ed.data_ptr())
    assert e.value.status == gsb.EINVAL
