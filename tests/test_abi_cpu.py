"""CPU-only checks of the C ABI: the library loads and exports every symbol
of include/hmat.h, argument validation fails cleanly without a GPU, and the
host-side cluster tree and block partition (Section 2.1) are identical to the
oracle's, bit for bit."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_2205_04752_gb300 import binding, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_functions():
    src = open(os.path.join(ROOT, "include", "hmat.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_\s\*]*?\b(hm_[a-z0-9_]+)\s*\(",
                       src, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_header_symbol():
    lib = binding.load()
    names = _header_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(binding.SYMBOLS)


def test_binding_constants_match_header():
    src = open(os.path.join(ROOT, "include", "hmat.h")).read()
    defs = dict(re.findall(r"^#define (HM_[A-Z0-9_]+) \(?(-?\d+)\)?", src, flags=re.M))
    assert int(defs["HM_MAX_LEAF"]) == binding.MAX_LEAF
    for name in ("HM_OK", "HM_EINVAL", "HM_ENOMEM", "HM_ENOTCONV", "HM_ETIMEOUT", "HM_EDEVICE", "HM_ERANK"):
        assert int(defs[name]) == getattr(binding, name), name
    for name, key in (("HM_FP64", "fp64"), ("HM_FP32", "fp32"), ("HM_BF16", "bf16"), ("HM_FP16", "fp16")):
        assert int(defs[name]) == binding.FORMS[key], name


def test_invalid_arguments_fail_cleanly():
    V, T = inputs.icosphere(1)
    with pytest.raises(binding.HMError) as e:
        binding.build_cluster_tree(V, T, 0, 0.8)
    assert e.value.code == binding.HM_EINVAL
    # the streamed product holds a leaf's rows in one CTA and one FP64
    # near-field column (6 x 336 values) in one 16 KB stage: at most 336
    binding.build_cluster_tree(V, T, 336, 0.8)
    with pytest.raises(binding.HMError) as e:
        binding.build_cluster_tree(V, T, 337, 0.8)
    assert b"336" in binding.load().hm_last_error()
    with pytest.raises(binding.HMError):
        binding.build_cluster_tree(V, T, 8, -1.0)
    bad = T.copy()
    bad[3, 1] = len(V) + 5
    with pytest.raises(binding.HMError):
        binding.build_cluster_tree(V, bad, 8, 0.8)
    deg = T.copy()
    deg[2] = [deg[2, 0], deg[2, 0], deg[2, 1]]
    with pytest.raises(binding.HMError):
        binding.build_cluster_tree(V, deg, 8, 0.8)
    Vn = V.copy()
    Vn[0, 0] = np.nan
    with pytest.raises(binding.HMError):
        binding.build_cluster_tree(Vn, T, 8, 0.8)
    # NULL pointers through the raw ABI
    lib = binding.load()
    out = ctypes.c_void_p()
    assert lib.hm_build_cluster_tree(None, 0, None, 0, 8, 0.8, ctypes.byref(out)) == binding.HM_EINVAL
    assert b"NULL" in lib.hm_last_error() or b"empty" in lib.hm_last_error()
    assert lib.hm_matvec(None, None, None, 1, 3, 0, None) == binding.HM_EINVAL
    assert lib.hm_pack(None, 1, None) == binding.HM_EINVAL
    assert lib.hm_amvm(None, None, None, None, None, None, None, 0, None, None) == binding.HM_EINVAL


def _compare_tree(V, T, leaf, eta):
    tr = binding.build_cluster_tree(V, T, leaf, eta)
    perm, nodes, adm, near = tr.export()
    Ho = oracle.HMatrix(V, T, leaf, eta, 1e-4)
    np.testing.assert_array_equal(perm, Ho.perm)
    np.testing.assert_array_equal(nodes, Ho.nodes)
    np.testing.assert_array_equal(adm, Ho.adm)
    np.testing.assert_array_equal(near, Ho.near)
    return tr


@pytest.mark.parametrize("mesh,leaf,eta", [
    ("ico0", 4, 0.8), ("ico3", 32, 0.8), ("ico3", 7, 0.8), ("ico4", 64, 0.5),
    ("cube6", 16, 0.8), ("ell", 32, 0.8), ("ico2", 336, 0.8)])
def test_tree_and_partition_match_oracle(mesh, leaf, eta):
    if mesh.startswith("ico"):
        V, T = inputs.icosphere(int(mesh[3:]))
    elif mesh == "cube6":
        V, T = inputs.cube_surface(6)
    else:
        V, T = inputs.ellipsoid(9, 0.6, 1.7, 1.1)
    tr = _compare_tree(V, T, leaf, eta)
    if leaf >= len(T):
        assert tr.nadm == 0 and tr.nnear == 1 and tr.nleaves == 1


@pytest.mark.slow
def test_tree_and_partition_match_oracle_level6():
    """The level-6 icosphere of the benchmark (81,920 triangles, leaf 64)."""
    V, T = inputs.icosphere(6)
    tr = _compare_tree(V, T, 64, 0.8)
    assert tr.nadm > 100000 and tr.nnear > 50000


@pytest.mark.parametrize("level,leaf,leaf_pts,npts,r_in,r_out", [
    (3, 32, 24, 700, 0.0, 0.95), (2, 16, 7, 333, 0.0, 0.7), (4, 64, 64, 2000, 0.0, 0.9),
    (1, 8, 1, 5, 0.0, 0.5), (2, 16, 32, 257, 1.2, 3.0), (2, 16, 336, 96, 0.0, 0.8)])
def test_point_tree_and_partition_match_oracle(level, leaf, leaf_pts, npts, r_in, r_out):
    """The rows of the evaluation operator (Section 5, Eq. (vector_eq)): the
    tree of the points and the partition (point tree) x (triangle tree) are
    the oracle's, bit for bit; the point tree outlives the triangle tree it
    was built from."""
    V, T = inputs.icosphere(level)
    P = inputs.shell_points(npts, r_in, r_out, 3)
    tr = binding.build_cluster_tree(V, T, leaf, 0.8)
    pt = binding.build_point_tree(tr, P, leaf_pts)
    del tr
    perm, nodes, adm, near = pt.export()
    Ho = oracle.HMatrix(V, T, leaf, 0.8, 1e-4, points=P, leaf_points=leaf_pts)
    np.testing.assert_array_equal(perm, Ho.rperm)
    np.testing.assert_array_equal(nodes, Ho.rnodes)
    np.testing.assert_array_equal(adm, Ho.adm)
    np.testing.assert_array_equal(near, Ho.near)
    assert pt.M == npts and pt.M_src == len(T)


def test_point_tree_invalid_arguments():
    V, T = inputs.icosphere(1)
    tr = binding.build_cluster_tree(V, T, 8, 0.8)
    P = inputs.ball_points(20, 0.5, 1)
    for leaf in (0, 337):
        with pytest.raises(binding.HMError) as e:
            binding.build_point_tree(tr, P, leaf)
        assert e.value.code == binding.HM_EINVAL
    Pn = P.copy()
    Pn[3, 2] = np.inf
    with pytest.raises(binding.HMError):
        binding.build_point_tree(tr, Pn, 8)
    with pytest.raises(binding.HMError):
        binding.build_point_tree(tr, P[:0], 8)
    pt = binding.build_point_tree(tr, P, 8)
    with pytest.raises(binding.HMError):
        binding.build_point_tree(pt, P, 8)  # a point tree is no surface
    lib = binding.load()
    out = ctypes.c_void_p()
    assert lib.hm_build_point_tree(None, None, 0, 8, ctypes.byref(out)) == binding.HM_EINVAL
    assert lib.hm_eval_points(None, None, None, 1, 0, None) == binding.HM_EINVAL
    assert lib.hm_baca(None, None, None, None, None, None, 0, None, None) == binding.HM_EINVAL


@pytest.mark.slow
def test_point_tree_and_partition_match_oracle_level6():
    """The evaluation operator's benchmark workload: 65,536 points in the ball
    of radius 0.95 inside the level-6 icosphere, leaves of 64 on both sides."""
    V, T = inputs.icosphere(6)
    P = inputs.ball_points(65536, 0.95, 7)
    tr = binding.build_cluster_tree(V, T, 64, 0.8)
    pt = binding.build_point_tree(tr, P, 64)
    perm, nodes, adm, near = pt.export()
    Ho = oracle.HMatrix(V, T, 64, 0.8, 1e-4, points=P, leaf_points=64)
    np.testing.assert_array_equal(perm, Ho.rperm)
    np.testing.assert_array_equal(nodes, Ho.rnodes)
    np.testing.assert_array_equal(adm, Ho.adm)
    np.testing.assert_array_equal(near, Ho.near)
    assert pt.nadm == 121407 and pt.nnear == 30638


@pytest.mark.parametrize("mesh,leaf,leaf_v", [("ico3", 32, 24), ("ico2", 16, 7), ("cube6", 16, 16),
                                              ("ico4", 64, 64), ("ico1", 8, 336)])
def test_vertex_tree_and_partition_match_oracle(mesh, leaf, leaf_v):
    """The columns of the double layer's K_Delta (Eq. (Kh)): the vertex tree
    with star boxes and the partition triangles x vertices equal the
    oracle's bit for bit; the blocks tile the M x nv rectangle, every vertex
    box holds the stars of its vertices, Eq. (adm) holds on every admissible
    block; the device assembly refuses the tree (not built)."""
    V, T = inputs.cube_surface(6) if mesh == "cube6" else inputs.icosphere(int(mesh[3:]))
    tr = binding.build_cluster_tree(V, T, leaf, 0.8)
    vt = binding.build_vertex_tree(tr, leaf_v)
    perm, nodes, adm, near = vt.export()
    op = oracle.VertexPartition(V, T, leaf, leaf_v, 0.8)
    np.testing.assert_array_equal(perm, op.perm)
    np.testing.assert_array_equal(nodes, op.nodes)
    np.testing.assert_array_equal(adm, op.adm)
    np.testing.assert_array_equal(near, op.near)
    assert vt.M == len(V) and vt.M_src == len(T)
    _, tnodes, _, _ = tr.export()
    cover = np.zeros((len(T), len(V)), dtype=np.int32)
    for (t, s) in np.concatenate([adm, near]):
        cover[tnodes[t, 0]:tnodes[t, 1], nodes[s, 0]:nodes[s, 1]] += 1
    assert np.all(cover == 1)
    for n in range(op.nnodes):
        lo, hi = nodes[n, 0], nodes[n, 1]
        verts = set(perm[lo:hi].tolist())
        tris = [i for i in range(len(T)) if verts & set(T[i].tolist())]
        pts = V[T[tris].reshape(-1)]
        assert np.all(op.boxes[n, :3] <= pts.min(0)) and np.all(op.boxes[n, 3:] >= pts.max(0))
        if n > 40:
            break
    # a vertex tree cannot stand in for a triangle tree (host checks, no GPU needed)
    with pytest.raises(binding.HMError):
        binding.build_point_tree(vt, inputs.ball_points(4, 0.5, 1), 8)
    with pytest.raises(binding.HMError):
        binding.build_vertex_tree(vt, 8)


def test_bench_script_parses_its_arguments():
    """bench.py imports and parses its flags on any host; the work itself
    needs a GPU."""
    import subprocess
    import sys
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--help"], capture_output=True, text=True,
                       timeout=120)
    assert r.returncode == 0, r.stderr
    for flag in ("--no-points", "--no-baca", "--points-minimal", "--impl"):
        assert flag in r.stdout
