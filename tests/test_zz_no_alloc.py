"""The no-allocation field solve (itokmc_field_solve_noalloc) against the
oracle's exact solve of the discrete Poisson problem and against the handle's
own field solve.

Callers that cannot call cudaMalloc (device memory owned by another runtime's
pool, code that must avoid the implicit synchronisation of cudaMalloc/
cudaFree, plugins whose host forbids new device allocations) use this entry
point: the library takes its multigrid scratch from a static device array and
the caller passes the charge, potential and field buffers.  Here the buffers
are torch tensors made by the test; the two paths must agree within the
field tolerance of the parity tests on two calls in a row.  This file is
named so that pytest collects it last.
"""
import numpy as np
import pytest

from oracle import poisson
from paper_2307_01797_gb300 import itokmc, synth

from gpu_util import gpu_handle, mixed_state, small_phys

pytestmark = pytest.mark.gpu

E_TOL = 1e-5


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("precision", [itokmc.FP64, itokmc.MIXED])
def test_noalloc_solve_matches_handle_two_calls(precision):
    import torch
    assert torch.cuda.is_available()
    ph = small_phys(32, dt=5e-12, photon_ratio=0.06)
    st = mixed_state(ph, seed=44, peak=2e18)
    ions = synth.random_ions(ph, seed=45, mean=400)
    H = gpu_handle(ph, 8 * len(st["w"]) + 100000, seed0=3, precision=precision)
    H.itokmc_set_particles(st["x"], st["y"], st["z"], st["w"])
    H.itokmc_set_ions(*ions)
    H.itokmc_solve_field()
    n3 = ph["n"] ** 3
    cfg = itokmc.make_config(ph, 1, precision=precision)
    cfg.stream = torch.cuda.current_stream().cuda_stream
    phi_d = torch.zeros(n3, dtype=torch.float64, device="cuda")
    E_d = torch.empty(3 * n3, dtype=torch.float64, device="cuda")
    for call in range(2):
        rho = H.itokmc_read_densities(itokmc.RHO)
        phi_ref = H.itokmc_read_densities(itokmc.PHI)
        E_ref = H.itokmc_read_densities(itokmc.E).ravel()
        rho_d = torch.from_numpy(rho).to("cuda")
        phi_d.zero_()
        cycles, rel = itokmc.itokmc_field_solve_noalloc(cfg, rho_d, phi_d, E_d)
        torch.cuda.synchronize()
        assert rel <= 1e-10 and cycles > 0
        # the exact solution of the discrete system (oracle, separable direct solve)
        phi_ex, E_ex = poisson.solve(rho, ph)
        E_ex = np.concatenate([np.asarray(b).ravel() for b in E_ex])
        assert _rel(phi_d.cpu().numpy(), np.asarray(phi_ex).ravel()) < E_TOL
        assert _rel(E_d.cpu().numpy(), E_ex) < E_TOL
        assert _rel(phi_d.cpu().numpy(), phi_ref) < E_TOL
        assert _rel(E_d.cpu().numpy(), E_ref) < E_TOL
        # the second call sees a new charge: one more step of the handle
        H.itokmc_step(1)


def test_noalloc_rejects_grids_beyond_its_scratch():
    ph = small_phys(128)
    cfg = itokmc.make_config(ph, 1)
    import torch
    z = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(itokmc.ItokmcError) as e:
        itokmc.itokmc_field_solve_noalloc(cfg, z, z, z)
    assert e.value.code == -1 and "64" in str(e.value)


@pytest.mark.parametrize("field", [(2, -1), (0, 2), (5, 0)])
def test_noalloc_rejects_unknown_precision(field):
    """A precision or field precision other than FP64 / MIXED (-1 for the
    field: as precision) is refused on the host before any launch."""
    import torch
    ph = small_phys(16)
    cfg = itokmc.make_config(ph, 1)
    cfg.precision, cfg.field_precision = field
    n3 = 16 ** 3
    rho = torch.zeros(n3, dtype=torch.int64, device="cuda")
    phi = torch.full((n3,), 7.0, dtype=torch.float64, device="cuda")
    E = torch.full((3 * n3,), 7.0, dtype=torch.float64, device="cuda")
    with pytest.raises(itokmc.ItokmcError) as e:
        itokmc.itokmc_field_solve_noalloc(cfg, rho, phi, E)
    assert e.value.code == -1 and "precision" in str(e.value)
    torch.cuda.synchronize()
    assert bool((phi == 7.0).all()) and bool((E == 7.0).all())
