"""Helpers of the GPU tests: run the CUDA path on seeded inputs and compare
with the FP64 oracle at the stated tolerances."""
from __future__ import annotations

import numpy as np

RHO_RTOL = 1e-5       # rho: all terms positive, plain relative tolerance
D_STOL = 1e-4         # drho/dh: |err| <= 1e-4 * S_i, S_i = sum_j m_j |dW/dh|


def torch_dev():
    import torch
    return torch.device("cuda", 0)


def run_density(boxes, uniform_mass=False, count_candidates=False, expect_flags=False,
                launch_shape=None):
    """Runs sort + density on one or more Box objects (concatenated);
    launch_shape = (density, adjoint) CTAs per SM, or None for the default."""
    import torch
    from paper_1804_06231_gb300.pv import Grid
    if not isinstance(boxes, (list, tuple)):
        boxes = [boxes]
    dev = torch_dev()
    pos = torch.from_numpy(np.concatenate([b.pos for b in boxes])).to(dev)
    h = torch.from_numpy(np.concatenate([b.h for b in boxes])).to(dev)
    m = torch.from_numpy(np.concatenate([b.m for b in boxes])).to(dev)
    with Grid([(b.n, b.L, b.nc) for b in boxes]) as g:
        if launch_shape:
            g.set_tuning(*launch_shape)
        if uniform_mass:
            g.sort(pos, h, None, m_uniform=float(boxes[0].m[0]))
        else:
            g.sort(pos, h, m)
        rho, D, n = g.density()
        cand = g.count_candidates() if count_candidates else None
        st = g.stats(raise_on_flags=False)
    torch.cuda.synchronize()
    if not expect_flags:
        assert st.device_flags == 0, f"device flags {st.device_flags}"

    # Widened on the device: with flags latched the outputs are unwritten, and
    # numpy warns when it widens arbitrary bit patterns.
    return (rho.double().cpu().numpy(), D.double().cpu().numpy(), n.cpu().numpy(), st, cand)


def check_density(rho, D, n, ref, idx=None):
    """Asserts the parity bar; idx selects the oracle particles compared."""
    if idx is not None:
        rho, D, n = rho[idx], D[idx], n[idx]
    rel = np.abs(rho / ref.rho - 1.0)
    assert rel.max() <= RHO_RTOL, f"rho max rel err {rel.max():.3e}"
    derr = np.abs(D - ref.drho_dh)
    assert np.all(derr <= D_STOL * ref.S), f"drho/dh max scaled err {(derr / ref.S).max():.3e}"
    exact = ref.band == 0
    assert np.array_equal(n[exact], ref.n_ngb[exact]), \
        f"n mismatch on {(n[exact] != ref.n_ngb[exact]).sum()} particles"
    assert np.all(np.abs(n[~exact] - ref.n_ngb[~exact]) <= ref.band[~exact])
