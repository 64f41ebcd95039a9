"""The FP32 certificate of the line search (Sec. 5.4): a row it certifies has psi(s) >= 0, evaluated
here in extended precision (numpy's long double) and by the FP64 formula the line search would otherwise
use; and it certifies nearly every comfortably feasible row, for small and for large relative density
changes |s A_rho / rho0| alike."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_04514_gb300 import build

    build.build()
    return torch


def _rows(rng, n, gamma, dim=2):
    rho = np.exp(rng.uniform(np.log(1e-3), np.log(1e3), n))
    p = np.exp(rng.uniform(np.log(1e-3), np.log(1e3), n))
    a = np.sqrt(gamma * p / rho)
    v = rng.normal(size=(dim, n))
    v *= rng.uniform(0, 5, n) * a / np.linalg.norm(v, axis=0)
    eps = p / (gamma - 1.0)
    E = eps + 0.5 * rho * (v * v).sum(0)
    U0 = np.concatenate([rho[None], rho * v, E[None]])
    st0 = rho ** (-gamma) * eps
    smin = st0 * (1.0 - np.exp(rng.uniform(np.log(1e-8), np.log(1e-1), n)))
    # A: a random direction with |A_q| ~ rel |U0_q| (rel log-uniform over [1e-8, 0.3])
    rel = np.exp(rng.uniform(np.log(1e-8), np.log(0.3), n))
    scale = np.abs(U0).max(0)
    A = rng.normal(size=U0.shape) * rel * scale
    A[0] = rng.normal(size=n) * rel * rho
    s = rng.uniform(0, 1, n)
    return np.concatenate([U0, A, smin[None], s[None]]).T.copy()


def _psi_ld(rows, gamma, dim=2):
    m = dim + 2
    r = rows.astype(np.longdouble)
    V = r[:, :m] + r[:, 2 * m + 1:2 * m + 2] * r[:, m:2 * m]
    rho = V[:, 0]
    eps = V[:, -1] - 0.5 * (V[:, 1:-1] ** 2).sum(1) / rho
    return eps - r[:, 2 * m] * np.power(rho, np.longdouble(gamma))


@pytest.mark.parametrize("gamma", [1.4, 5.0 / 3.0])
def test_certified_rows_are_feasible(torch_cuda, gamma):
    torch = torch_cuda
    from paper_2402_04514_gb300.gdg import certificate_check

    rng = np.random.default_rng(5)
    rows = _rows(rng, 300000, gamma)
    out = certificate_check(2, gamma, torch.from_numpy(rows).cuda()).cpu().numpy()
    cert = out[:, 0] == 1.0
    psi64 = out[:, 1]
    psi = _psi_ld(rows, gamma)
    assert (psi[cert] >= 0).all() and (psi64[cert] >= 0).all()
    x = np.abs(rows[:, 9] * rows[:, 4] / rows[:, 0])  # s A_rho / rho0
    eps0 = rows[:, 3] - 0.5 * (rows[:, 1] ** 2 + rows[:, 2] ** 2) / rows[:, 0]
    easy = psi.astype(np.float64) > 0.01 * eps0
    for branch, sel in (("|x| <= 1/16", x <= 1.0 / 16), ("|x| > 1/16", x > 1.0 / 16)):
        rate = cert[easy & sel].mean()
        print(f"gamma {gamma} {branch}: {(easy & sel).sum()} comfortably feasible rows, certified {rate:.4f}")
        assert (easy & sel).sum() > 1000 and rate > 0.99


@pytest.mark.parametrize("gamma", [1.4, 5.0 / 3.0])
def test_increments_below_fp32_range(torch_cuda, gamma):
    """Components of A below the FP32 normal range (|A_q| < 2^-126, rounding residuals of a uniform
    neighbourhood) count as 0 when s |A_q| is below half an ulp of U0_q: the FP64 search then evaluates
    psi at the same point as for A_q = 0, so the certificate decides both alike.  Where U0_q is 0 the guard
    cannot hold and the row is not certified."""
    torch = torch_cuda
    from paper_2402_04514_gb300.gdg import certificate_check

    rng = np.random.default_rng(11)
    n, m = 200000, 4
    rows = _rows(rng, n, gamma)
    tiny = rng.random((n, m)) < 0.5
    mag = np.exp(rng.uniform(np.log(1e-300), np.log(1e-39), (n, m))) * rng.choice([-1.0, 1.0], (n, m))
    A = rows[:, m:2 * m]
    A[tiny] = mag[tiny]
    flushed = rows.copy()
    flushed[:, m:2 * m][tiny] = 0.0
    out = certificate_check(2, gamma, torch.from_numpy(rows).cuda()).cpu().numpy()
    ref = certificate_check(2, gamma, torch.from_numpy(flushed).cuda()).cpu().numpy()
    assert np.array_equal(out[:, 1], ref[:, 1])  # the FP64 evaluation point does not see them
    assert np.array_equal(out[:, 0], ref[:, 0])
    assert out[:, 0].sum() > 10000
    psi = _psi_ld(rows, gamma)
    assert (psi[out[:, 0] == 1.0] >= 0).all()
    # a zero momentum component with a tiny increment: no guard, no certificate
    z = rows[:2000].copy()
    z[:, 1] = 0.0
    z[:, m + 1] = 1e-40
    out_z = certificate_check(2, gamma, torch.from_numpy(z).cuda()).cpu().numpy()
    assert (out_z[:, 0] == 0.0).all()
