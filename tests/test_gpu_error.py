"""Averaged-error evaluator on the GPU (Eq. (averageerror) and the bound of Eq.
(errorestimate)) against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1802_10291_gb300 import mci

pytestmark = pytest.mark.gpu

F, H, D1, D2 = ("identity",), ("hilbert",), ("deriv", 1), ("deriv", 2)


@pytest.mark.parametrize("systems,P", [([F], 32), ([F, D1], 16), ([F, H, D1], 32), ([F, D1, D2], 12),
                                       ([F, ("shift", 0.3)], 16), ([F, H], 64)])
def test_averaged_error_matches_oracle(cuda_device, systems, P):
    rng = np.random.default_rng(len(systems) * 100 + P)
    M = len(systems)
    n_max = 10 * M * P
    n = np.arange(-n_max, n_max + 1)
    batch = 5
    coeffs = []
    for b in range(batch):
        decay = 1.5 + 0.5 * b
        c = (rng.standard_normal(n.size) + 1j * rng.standard_normal(n.size)) / (1.0 + np.abs(n)) ** decay
        coeffs.append(c)
    C = np.stack(coeffs)
    d = torch.tensor(np.stack([C.real, C.imag], -1).reshape(batch, -1), dtype=torch.float64, device="cuda")
    eps = torch.empty(batch, dtype=torch.float64, device="cuda")
    bnd = torch.empty(batch, dtype=torch.float64, device="cuda")
    plan = mci.Plan(systems, P, 4 * P, max_batch=1)
    mci.mci_averaged_error(plan.handle, 0, d, n_max, batch, eps, bnd)
    torch.cuda.synchronize()
    e, bb = eps.cpu().numpy(), bnd.cpu().numpy()
    for b in range(batch):
        tab = dict(zip(n.tolist(), C[b]))
        fn = lambda k: np.array([tab.get(int(v), 0.0) for v in np.atleast_1d(k)])
        ref = O.averaged_error(fn, systems, P, n_max=n_max)
        refb = O.error_bound(fn, systems, P, n_max=n_max)
        assert abs(e[b] - ref) <= 1e-12 * ref, (e[b], ref)
        assert abs(bb[b] - refb) <= 1e-12 * refb, (bb[b], refb)
        assert bb[b] >= e[b] * (1 - 1e-12)
    plan.close()


def test_bandlimited_signal_has_zero_error(cuda_device):
    systems, P = [F, H, D1], 32
    n_max = 400
    n = np.arange(-n_max, n_max + 1)
    N1 = -(3 * P) // 2
    c = np.where((n >= N1) & (n < N1 + 3 * P), 1.0 / (1.0 + np.abs(n)), 0.0).astype(np.complex128)
    d = torch.tensor(np.stack([c.real, c.imag], -1).reshape(1, -1), dtype=torch.float64, device="cuda")
    eps = torch.empty(1, dtype=torch.float64, device="cuda")
    plan = mci.Plan(systems, P, 4 * P, max_batch=1)
    mci.mci_averaged_error(plan.handle, 0, d, n_max, 1, eps)
    torch.cuda.synchronize()
    assert eps.item() == 0.0
    plan.close()


def test_averaged_error_argument_checks(cuda_device):
    plan = mci.Plan([F, D1], 16, 64, channels="fd", max_batch=1)
    d = torch.zeros(2 * 401, dtype=torch.float64, device="cuda")
    eps = torch.empty(1, dtype=torch.float64, device="cuda")
    with pytest.raises(mci.MciError):
        mci.mci_averaged_error(plan.handle, 0, d, 200, 1, eps)      # FD channels
    plan.close()
    plan = mci.Plan([F, D1], 16, 64, max_batch=1)
    with pytest.raises(mci.MciError):
        mci.mci_averaged_error(plan.handle, 0, d, 10, 1, eps)       # n_max inside the band
    with pytest.raises(mci.MciError):
        mci.mci_averaged_error(plan.handle, 1, d, 200, 1, eps)      # no such class
    plan.close()
