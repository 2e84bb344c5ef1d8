"""Shared helpers for the GPU parity tests (inputs from meshgen, expected values from the oracle)."""
import numpy as np

import oracle

W_TOL = 1e-4        # |w_gpu - w_fp64| for queries farther than NEAR from the surface
NEAR = 1e-3         # distance that selects FP64 re-evaluation
TIE = 1e-9          # |w_fp64 - 0.5| below this is a tie: either occupancy is accepted
GRAD_REL = 1e-3     # relative Frobenius error of dL/dV


def to_dev(a, dev):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def make_mesh(V, F, dev):
    from paper_2407_11272_b300 import dv

    return dv.dv_mesh_create(to_dev(V, dev), to_dev(F, dev))


def oracle_grid(V, F, grid, with_distance=True):
    Q = oracle.grid_queries(grid.lo, grid.hi, grid.n)
    w = oracle.winding(V, F, Q)
    d = oracle.point_mesh_distance(V, F, Q) if with_distance else None
    return Q, w, d


def check_forward(w_gpu, w64, d, prec, occ_gpu=None, label=""):
    """Assert the forward parity bar; returns a dict of error statistics."""
    w_gpu = np.asarray(w_gpu, dtype=np.float64)
    far = d > NEAR
    err = np.abs(w_gpu - w64)
    stats = {"max_err_far": float(err[far].max()) if far.any() else 0.0, "n_far": int(far.sum())}
    assert stats["max_err_far"] <= W_TOL, f"{label} {prec}: max |dw| far from surface {stats['max_err_far']:.3e}"
    assert np.all(np.isfinite(w_gpu)), f"{label}: non-finite w"
    if prec == "mixed":
        # every near-surface query went through FP64: w matches to FP32 output rounding
        near = ~far
        if near.any():
            stats["max_err_near"] = float(err[near].max())
            assert stats["max_err_near"] <= 1e-6 * max(1.0, np.abs(w64[near]).max()), \
                f"{label}: near-surface |dw| {stats['max_err_near']:.3e} (not re-evaluated in FP64?)"
        if occ_gpu is not None:
            occ64 = (w64 > 0.5).astype(np.uint8)
            tie = np.abs(w64 - 0.5) <= TIE
            bad = (np.asarray(occ_gpu) != occ64) & ~tie
            assert not bad.any(), f"{label}: {bad.sum()} occupancy mismatches after re-evaluation"
    elif occ_gpu is not None:
        occ64 = (w64 > 0.5).astype(np.uint8)
        safe = far & (np.abs(w64 - 0.5) > 1e-3)
        bad = (np.asarray(occ_gpu) != occ64) & safe
        assert not bad.any(), f"{label}: {bad.sum()} occupancy mismatches away from the threshold"
    return stats


CANCEL = 1e-5      # FP32 per-vertex error allowed relative to the sum of |face contributions|


def grad_close(G_gpu, G_ref, label="", scale=None):
    """Relative Frobenius error and a per-vertex criterion for dL/dV.

    Per vertex: |dG_v| <= GRAD_REL * max(|G_v|, 1e-2 rms) + CANCEL * scale_v, where scale_v is
    the sum over the vertex's faces of |face contribution| (oracle.winding_grad_scale): where the
    faces' contributions cancel (vertices away from the holes of an open mesh have an exact
    gradient of 0), FP32 can only be held to a fraction of the terms that cancel."""
    G_gpu = np.asarray(G_gpu, dtype=np.float64)
    diff = np.linalg.norm(G_gpu - G_ref)
    ref = np.linalg.norm(G_ref)
    rel = diff / max(ref, 1e-300)
    assert rel <= GRAD_REL, f"{label}: relative Frobenius error {rel:.3e}"
    rms = np.sqrt(np.mean(np.sum(G_ref ** 2, axis=1)))
    per = np.linalg.norm(G_gpu - G_ref, axis=1)
    lim = GRAD_REL * np.maximum(np.linalg.norm(G_ref, axis=1), 1e-2 * rms)
    if scale is not None:
        lim = lim + CANCEL * np.asarray(scale)
    bad = per > lim
    assert not bad.any(), (f"{label}: {bad.sum()} vertices outside the per-vertex bound; worst: "
                           f"|dG|={per[bad].max():.3e} |G|={np.linalg.norm(G_ref, axis=1)[bad].max():.3e} "
                           f"rms={rms:.3e} scale={(np.asarray(scale)[bad].max() if scale is not None else 0):.3e}")
    return rel
