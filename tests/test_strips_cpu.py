"""Strip order of the faces (dv_build_strips, a host function of the library; no GPU).

The forward passes visit faces in this order and take |v - q| of a face's older vertices and
the dot of its older edge from the events before it, so the order must (1) contain every face
exactly once, (2) give each face event the face's own vertex set as its last three vertices,
and (3) actually share vertices (events per face well below 3) on the benchmark meshes."""
import numpy as np
import pytest

from paper_2407_11272_b300 import dv, meshgen


def _check_order(F, ev_vert, ev_face):
    nf = len(F)
    assert ev_vert.shape == ev_face.shape
    assert nf <= len(ev_vert) <= 3 * nf
    faces_seen = ev_face[ev_face >= 0]
    assert np.array_equal(np.sort(faces_seen), np.arange(nf)), "every face exactly once"
    k = 0
    n = len(ev_vert)
    while k < n:
        # a strip: two vertex-only events, then at least one face event
        assert k + 2 < n and ev_face[k] == -1 and ev_face[k + 1] == -1 and ev_face[k + 2] >= 0, k
        k += 2
        while k < n and ev_face[k] >= 0:
            f = ev_face[k]
            assert sorted(ev_vert[k - 2:k + 1].tolist()) == sorted(F[f].tolist()), (k, f)
            k += 1


@pytest.mark.parametrize("kind", ["torus", "icosphere", "sh_sphere", "open_sheet"])
def test_strip_order_valid(kind):
    if kind == "torus":
        V, F = meshgen.jittered_torus()
    elif kind == "icosphere":
        V, F = meshgen.icosphere(3, 0.8)
    elif kind == "sh_sphere":
        V, F = meshgen.sh_sphere(freq=20)
    else:
        V, F = meshgen.jittered_torus(nu=12, nv=7, sigma=0.0, delete_frac=0.4, seed=3)
    ev_vert, ev_face = dv.dv_build_strips(F, len(V))
    _check_order(F, ev_vert, ev_face)
    per_face = len(ev_vert) / len(F)
    if kind == "torus":
        assert per_face < 1.3, per_face  # 10 % faces deleted: strips break at the holes
    if kind in ("icosphere", "sh_sphere"):
        assert per_face < 1.1, per_face


def test_strip_order_odd_inputs():
    # non-manifold edge (three faces on edge 0-1), a degenerate face, an isolated face, and
    # two faces with opposite orientations across an edge
    F = np.array([[0, 1, 2], [1, 0, 3], [0, 1, 4], [5, 5, 6], [7, 8, 9], [2, 1, 10], [2, 10, 11]], dtype=np.int32)
    ev_vert, ev_face = dv.dv_build_strips(F, 12)
    _check_order(F, ev_vert, ev_face)
    one = np.array([[0, 1, 2]], dtype=np.int32)
    ev_vert, ev_face = dv.dv_build_strips(one, 3)
    assert sorted(ev_vert.tolist()) == [0, 1, 2] and ev_face.tolist() == [-1, -1, 0]


def test_strip_order_errors():
    F = np.array([[0, 1, 2], [0, 2, 5]], dtype=np.int32)
    with pytest.raises(dv.DvError):
        dv.dv_build_strips(F, 5)  # index 5 outside [0, 5)
    with pytest.raises(dv.DvError):
        dv.dv_build_strips(np.array([[0, -1, 2]], dtype=np.int32), 3)


def test_strip_order_deterministic():
    V, F = meshgen.jittered_torus(nu=40, nv=20, sigma=0.01, delete_frac=0.1, seed=2)
    a = dv.dv_build_strips(F, len(V))
    b = dv.dv_build_strips(F, len(V))
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def _check_pairs(F, pairs, singles):
    """Every face in exactly one pair or in singles; each pair's records describe its two faces:
    A = (p0, p1, p2) is a rotation of fA's corners and the code maps its canonical corners onto
    them; B = (p2, p1, p3) is fB's vertex set, its corners mapped by the code, with bit 12 set
    exactly when (p2, p1, p3) is not a rotation of fB's corners."""
    nf = len(F)
    seen = np.concatenate([pairs[:, 4], pairs[:, 5], singles]) if len(pairs) else singles
    assert np.array_equal(np.sort(seen), np.arange(nf)), "every face exactly once"
    assert np.all(pairs[:, 7] == 0)
    for p0, p1, p2, p3, fa, fb, code, _ in pairs.tolist():
        assert len({p0, p1, p2, p3}) == 4
        ca = [(code >> (2 * c)) & 3 for c in range(3)]
        cb = [(code >> (6 + 2 * c)) & 3 for c in range(3)]
        assert sorted(ca) == [0, 1, 2] and sorted(cb) == [0, 1, 2]
        assert [F[fa][ca[c]] for c in range(3)] == [p0, p1, p2]
        assert [F[fb][cb[c]] for c in range(3)] == [p2, p1, p3]
        # canonical A keeps fA's orientation: its corner map is a rotation
        assert ca in ([0, 1, 2], [1, 2, 0], [2, 0, 1])
        rot_b = cb in ([0, 1, 2], [1, 2, 0], [2, 0, 1])
        assert bool((code >> 12) & 1) == (not rot_b)
        assert code >> 13 == 0


@pytest.mark.parametrize("kind", ["torus", "icosphere", "odd"])
def test_face_pairs_valid(kind):
    if kind == "torus":
        V, F = meshgen.jittered_torus()
    elif kind == "icosphere":
        V, F = meshgen.icosphere(3, 0.8)
    else:
        V = np.zeros((12, 3), np.float32)
        F = np.array([[0, 1, 2], [1, 0, 3], [0, 1, 4], [5, 5, 6], [7, 8, 9], [2, 1, 10], [2, 10, 11],
                      [1, 2, 10]], dtype=np.int32)
    pairs, singles = dv.dv_build_face_pairs(F, len(V))
    _check_pairs(F, pairs, singles)
    if kind == "icosphere":
        assert 2 * len(pairs) >= 0.9 * len(F)  # long strips: nearly every face paired
    if kind == "torus":
        assert 2 * len(pairs) >= 0.7 * len(F)
    if kind == "odd":
        # the degenerate face [5, 5, 6] and the isolated face [7, 8, 9] stay single
        assert 3 in singles and 4 in singles


def test_face_pairs_reversed_orientation():
    """Two faces crossing their shared edge in the same direction (inconsistent orientation):
    they still pair, with bit 12 of the code set; randomly flipped torus faces give both kinds."""
    F = np.array([[0, 1, 2], [1, 2, 3]], dtype=np.int32)
    pairs, singles = dv.dv_build_face_pairs(F, 4)
    _check_pairs(F, pairs, singles)
    assert len(pairs) == 1 and len(singles) == 0 and (pairs[0, 6] >> 12) & 1 == 1
    V, F = meshgen.jittered_torus(nu=40, nv=20, sigma=0.01, delete_frac=0.1, seed=2)
    flip = np.random.default_rng(5).random(len(F)) < 0.3
    F[flip] = F[flip][:, ::-1]
    pairs, singles = dv.dv_build_face_pairs(F, len(V))
    _check_pairs(F, pairs, singles)
    rev = (pairs[:, 6] >> 12) & 1
    assert 0 < rev.sum() < len(pairs)


def test_face_pairs_random_meshes():
    """Random face sets over small vertex sets (shared, non-manifold, repeated and degenerate
    faces, both orientations): the pairing invariants hold on every one."""
    rng = np.random.default_rng(123)
    for trial in range(60):
        nv = int(rng.integers(3, 40))
        nf = int(rng.integers(1, 120))
        F = rng.integers(0, nv, size=(nf, 3)).astype(np.int32)
        pairs, singles = dv.dv_build_face_pairs(F, nv)
        _check_pairs(F, pairs, singles)
        ev_vert, ev_face = dv.dv_build_strips(F, nv)
        _check_order(F, ev_vert, ev_face)
    # a closed surface with consistently oriented faces: every pair is consistent (no bit 12)
    V, F = meshgen.icosphere(2, 0.7)
    pairs, _ = dv.dv_build_face_pairs(F, len(V))
    assert np.all(((pairs[:, 6] >> 12) & 1) == 0)


def test_face_pairs_argument_errors():
    """Host entry points reject bad arguments with the documented status codes."""
    import ctypes

    lib = dv.load()
    F = np.array([[0, 1, 2], [1, 2, 3]], dtype=np.int32)
    n_p, n_s = ctypes.c_int64(0), ctypes.c_int64(0)
    ptr = ctypes.c_void_p(F.ctypes.data)
    assert lib.dv_build_face_pairs(ptr, 2, 2, None, None, 0, 0, ctypes.byref(n_p), ctypes.byref(n_s)) == 1  # nv < 3
    assert lib.dv_build_face_pairs(None, 2, 4, None, None, 0, 0, ctypes.byref(n_p), ctypes.byref(n_s)) == 1
    bad = np.array([[0, 1, 9]], dtype=np.int32)
    assert lib.dv_build_face_pairs(ctypes.c_void_p(bad.ctypes.data), 1, 4, None, None, 0, 0, ctypes.byref(n_p),
                                   ctypes.byref(n_s)) == 2  # index outside [0, nv)
    assert lib.dv_build_face_pairs(ptr, 2, 4, None, None, 0, 0, ctypes.byref(n_p), ctypes.byref(n_s)) == 0
    assert (n_p.value, n_s.value) == (1, 0)
    out_p = np.zeros((1, 8), np.int32)
    out_s = np.zeros(1, np.int32)
    # a capacity below the count
    assert lib.dv_build_face_pairs(ptr, 2, 4, ctypes.c_void_p(out_p.ctypes.data), ctypes.c_void_p(out_s.ctypes.data),
                                   0, 1, ctypes.byref(n_p), ctypes.byref(n_s)) == 1
