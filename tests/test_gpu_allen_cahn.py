"""GPU parity of the Allen-Cahn pieces (Example 4) against the oracle: the TT
Laplacian and linear combination exactly, a few explicit Euler steps against
the oracle's steps, and on the full configuration (d = 8, n = 64) the decay
of the discrete energy."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import allen_cahn as oac
from oracle import tt as ott

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module")
def B():
    from paper_2410_04385_gb300 import binding, build
    if not os.path.exists(binding.LIB_PATH):
        build.build()
    binding.load()
    return binding


def to_gpu(cores):
    return [torch.from_numpy(np.ascontiguousarray(c)).cuda() for c in cores]


def to_np(cores):
    return [c.detach().cpu().numpy() for c in cores]


@pytest.mark.parametrize("d", [1, 2, 5])
def test_laplacian_matches_oracle(B, d):
    rng = np.random.default_rng(d)
    u = [rng.standard_normal((1 if k == 0 else 4, 9, 1 if k == d - 1 else 3 + (k % 2)))
         for k in range(d)]
    for k in range(1, d):
        u[k] = rng.standard_normal((u[k - 1].shape[2], 9, u[k].shape[2]))
    h = 0.37
    L = to_np(B.tt_laplacian(to_gpu(u), 1.0 / (h * h)))
    Lo = oac.laplacian_tt(u, h)
    assert [c.shape for c in L] == [c.shape for c in Lo]
    for a, b in zip(L, Lo):
        assert np.allclose(a, b, rtol=1e-14, atol=1e-12 * np.abs(b).max())


@pytest.mark.parametrize("d", [1, 3])
def test_lincomb_matches_oracle(B, d):
    rng = np.random.default_rng(10 + d)
    def tt(r):
        rk = [1] + [r] * (d - 1) + [1]
        return [rng.standard_normal((rk[k], 6, rk[k + 1])) for k in range(d)]
    T = [tt(1), tt(2), tt(3)]
    coef = [1.5, -0.25, 2.0]
    S = to_np(B.tt_lincomb([to_gpu(t) for t in T], coef))
    So = oac.lincomb_tt(T, coef)
    for a, b in zip(S, So):
        assert np.array_equal(a.shape, b.shape) and np.allclose(a, b, rtol=1e-15, atol=1e-15)


def test_steps_match_oracle(B):
    """d = 3, n = 8: every bond rank is at most 8, so no rank cap binds and
    the sketches are exact; the only truncation is the 1e-12 tolerance, and
    five GPU steps equal five oracle steps to that level. (With binding caps
    the two sides truncate near-equal singular values differently, and the
    oracle's rounding sweeps in the mirror order, so that comparison would
    measure the cap's sensitivity, not the kernels.)"""
    from paper_2410_04385_gb300 import allen_cahn as ac
    d, n, eps, dt = 3, 8, 0.1, 1e-3
    h = 2 * np.pi / n
    u = oac.initial_condition(d, n, seed=3)
    ug = to_gpu(u)
    for w in range(5):
        ug, _ = ac.step(ug, h, eps, dt, max_rank=64, tol=1e-12, hatt_tol=0.0, seed=100 * w)
        u, _ = oac.step(u, h, eps, dt, max_rank=64, tol=1e-12, hatt_tol=0.0, seed=100 * w)
    X = to_np(ug)
    assert ott.tt_diff_norm(X, u) <= 1e-10 * ott.tt_norm(u)


def test_full_configuration_energy_decays(B):
    """d = 8, n = 64, eps = 0.1, dt = 1e-3: 20 steps, energy non-increasing,
    ranks within the caps, no device wait ran out."""
    from paper_2410_04385_gb300 import allen_cahn as ac
    d, n, eps, dt = 8, 64, 0.1, 1e-3
    h = 2 * np.pi / n
    u = to_gpu(oac.initial_condition(d, n, seed=0))
    energies = []
    for w in range(20):
        u, u2 = ac.step(u, h, eps, dt, max_rank=24, tol=1e-8, hatt_tol=1e-10, seed=10 * w)
        energies.append(ac.energy(u, u2, h, eps))
    assert all(np.isfinite(energies))
    assert all(b <= a * (1 + 1e-9) for a, b in zip(energies, energies[1:]))
    assert max(c.shape[2] for c in u) <= 24
    assert B.device_error() == 0


def _pad_np(u, rank):
    rk = [1] + [max(c.shape[2], rank) for c in u[:-1]] + [1]
    out = []
    for k, c in enumerate(u):
        p = np.zeros((rk[k], c.shape[1], rk[k + 1]))
        p[: c.shape[0], :, : c.shape[2]] = c
        out.append(p)
    return out


def test_fixed_rank_graph_matches_oracle(B):
    """d = 3, n = 8, every bond held at rank 8 (the largest these modes allow):
    five steps (the capture's warm-up step and four graph replays) against five
    oracle steps with the same sketch seeds, the oracle's result padded back
    to rank 8 after every step so both sides sketch the same shapes."""
    from paper_2410_04385_gb300 import allen_cahn as ac
    d, n, eps, dt = 3, 8, 0.1, 1e-3
    h = 2 * np.pi / n
    u0 = _pad_np(oac.initial_condition(d, n, seed=3), 8)
    st = ac.FixedRankStepper(to_gpu(u0), h, eps, dt, rank=8, tol=1e-12, hatt_tol=0.0,
                             hatt_rank=8, seed=100)
    st.capture()
    for _ in range(4):
        st.replay()
    torch.cuda.synchronize()
    assert [c.shape for c in st.u] == [c.shape for c in u0]
    u = u0
    for _ in range(5):
        u, _ = oac.step(u, h, eps, dt, max_rank=8, tol=1e-12, hatt_tol=0.0, seed=100)
        u = _pad_np(u, 8)
    X = to_np(st.u)
    assert ott.tt_diff_norm(X, u) <= 1e-10 * ott.tt_norm(u)


def test_fixed_rank_graph_equals_eager_steps(B):
    """The captured step replays exactly what the eager step does."""
    from paper_2410_04385_gb300 import allen_cahn as ac
    d, n, eps, dt = 4, 16, 0.1, 1e-3
    h = 2 * np.pi / n
    u0 = to_gpu(oac.initial_condition(d, n, seed=5))
    a = ac.FixedRankStepper(u0, h, eps, dt, rank=12, tol=1e-8, hatt_tol=1e-10, hatt_rank=12,
                            seed=7)
    b = ac.FixedRankStepper(u0, h, eps, dt, rank=12, tol=1e-8, hatt_tol=1e-10, hatt_rank=12,
                            seed=7)
    for _ in range(4):
        a.step()
    b.capture()
    for _ in range(3):
        b.replay()
    torch.cuda.synchronize()
    for x, y in zip(a.u, b.u):
        assert torch.allclose(x, y, rtol=0.0, atol=1e-13 * float(y.abs().max()))


def test_fixed_rank_graph_full_configuration(B):
    """d = 8, n = 64 held at rank 24: 20 graph-replayed steps, energy
    non-increasing, no device wait ran out."""
    from paper_2410_04385_gb300 import allen_cahn as ac
    d, n, eps, dt = 8, 64, 0.1, 1e-3
    h = 2 * np.pi / n
    st = ac.FixedRankStepper(to_gpu(oac.initial_condition(d, n, seed=0)), h, eps, dt, rank=24,
                             tol=1e-8, hatt_tol=1e-10, hatt_rank=24, seed=10)
    st.capture()
    energies = []
    for _ in range(20):
        st.replay()
        torch.cuda.synchronize()
        energies.append(st.energy())
    assert all(np.isfinite(energies))
    assert all(b <= a * (1 + 1e-9) for a, b in zip(energies, energies[1:]))
    assert B.device_error() == 0
