"""Host logic of the request server on CPU: the served workload's statistics and the
memory-admission accounting (no GPU)."""
import math

import numpy as np
import pytest

from paper_2407_11272_b300.serve import GRID_SIZES, Admission, estimate_bytes, make_workload


def test_workload_matches_the_served_stream_description():
    reqs = make_workload(160, rate=200.0, seed=5)
    gaps = np.diff([0.0] + [r.arrival for r in reqs])
    assert np.all(gaps >= 0)
    assert 1 / 400 < gaps.mean() < 1 / 100  # Poisson at 200 req/s
    F = np.array([len(r.faces) for r in reqs])
    assert F.min() >= 20 and F.max() <= 2e5
    logs = np.log(F)
    assert math.log(500) - 1 < logs.mean() < math.log(1e5) + 1
    assert {r.n for r in reqs} <= set(GRID_SIZES) and len({r.n for r in reqs}) == len(GRID_SIZES)
    frac = np.mean([r.want_grad for r in reqs])
    assert 0.15 < frac < 0.45
    for r in reqs[:10]:
        assert r.faces.min() >= 0 and r.faces.max() < len(r.verts)
    # seeded: the same stream twice
    again = make_workload(5, rate=200.0, seed=5)
    assert all(np.array_equal(a.faces, b.faces) and a.arrival == b.arrival for a, b in zip(reqs, again))


def test_admission_respects_budget_and_fifo():
    adm = Admission(1000)
    assert adm.can_admit(5000)  # nothing in flight: even an oversize request may run alone
    adm.admit(600)
    assert adm.can_admit(400) and not adm.can_admit(401)
    adm.admit(400)
    assert not adm.can_admit(1)
    adm.release(600)
    assert adm.can_admit(600) and adm.used == 400
    adm.release(400)
    assert adm.used == 0 and adm.count == 0
    with pytest.raises(AssertionError):
        adm.release(1)


def test_estimate_grows_with_size():
    a = estimate_bytes(1000, 2000, 32, False)
    assert estimate_bytes(1000, 2000, 64, False) > a
    assert estimate_bytes(1000, 20000, 32, False) > a
    assert estimate_bytes(1000, 2000, 32, True) > a


def test_laplacian_energy_matches_autograd():
    """The morphing loop's gather-only Laplacian energy equals mean |L V|^2 of the scatter-add
    Laplacian, and its backward equals autograd's gradient of that expression (FP64, CPU)."""
    import torch

    from paper_2407_11272_b300 import meshgen
    from paper_2407_11272_b300.morph import LaplacianEnergy, laplacian, neighbour_table, uniform_laplacian_edges

    V0, F = meshgen.jittered_torus(nu=12, nv=7, sigma=0.02, delete_frac=0.2, seed=1)
    V = torch.from_numpy(V0.astype(np.float64))
    edges, deg = uniform_laplacian_edges(F, len(V0))
    nbr, w, wt = (torch.from_numpy(a) for a in neighbour_table(F, len(V0)))
    w, wt = w.double(), wt.double()
    Va = V.clone().requires_grad_(True)
    ref = laplacian(Va, torch.from_numpy(edges).long(), torch.from_numpy(deg).double()).pow(2).sum(dim=1).mean()
    ref.backward()
    Vb = V.clone().requires_grad_(True)
    E = LaplacianEnergy.apply(Vb, nbr, w, wt)
    E.backward()
    # the table's weights 1/deg are FP32 values: agreement to their rounding
    assert abs(float(E.detach()) - float(ref.detach())) <= 1e-6 * abs(float(ref.detach()))
    assert torch.allclose(Vb.grad, Va.grad, rtol=1e-6, atol=1e-9)
