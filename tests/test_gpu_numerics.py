"""The library's own FP64 reciprocal (hardware estimate + Newton-Raphson) held
against IEEE division on the same GPU."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_reciprocal_within_one_ulp_of_ieee_division(cuda_device):
    import torch
    from paper_2504_08157_gb300 import build, xg
    build.build()
    rng = np.random.default_rng(11)
    x = np.concatenate([
        rng.uniform(0.05, 2.0, 200000),                 # densities of the workloads
        np.exp(rng.uniform(-300.0, 300.0, 200000) * np.log(2.0)),   # wide exponent range
        np.array([1.0, 2.0, 0.5, 1.0 + 2.0 ** -52, 2.0 - 2.0 ** -52, 1.2345678901234567]),
    ])
    xd = torch.from_numpy(x).to(cuda_device)
    out = torch.empty_like(xd)
    xg.xg_reciprocal(xd, out)
    ieee = 1.0 / xd
    torch.cuda.synchronize()
    r, ref = out.cpu().numpy(), ieee.cpu().numpy()
    ulp = np.abs(r - ref) / np.spacing(ref)
    assert np.max(ulp) <= 1.0, np.max(ulp)
    assert np.mean(r == ref) > 0.99
