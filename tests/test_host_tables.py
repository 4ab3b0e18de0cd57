"""The library's host tables (csrc/tables.cpp: quadrature rules, DG and geometry bases at the
volume points) against the oracle's, on the CPU: tables.cpp is compiled with a small probe
(tests/native/tables_probe.cpp) under the library's host flags, and its output compared with the
oracle's rules and bases for every element family the device takes."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle.basis import gauss_legendre, gll_nodes, equispaced_nodes
from oracle import simplex, simplex3

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _cuda_include():
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "include", "cuda_runtime.h")):
            return os.path.join(c, "include")
    nv = shutil.which("nvcc")
    if nv:
        inc = os.path.join(os.path.dirname(os.path.dirname(nv)), "include")
        if os.path.exists(os.path.join(inc, "cuda_runtime.h")):
            return inc
    return None


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    inc = _cuda_include()
    if shutil.which("g++") is None or inc is None:
        pytest.skip("g++ or the CUDA headers not available")
    exe = str(tmp_path_factory.mktemp("probe") / "tables_probe")
    subprocess.run(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-I", inc, "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "native", "tables_probe.cpp"),
                    os.path.join(ROOT, "paper_1810_11080_gb300", "csrc", "tables.cpp"), "-o", exe],
                   check=True, capture_output=True, text=True)

    def run(fam, p, r):
        out = subprocess.run([exe, fam, str(p), str(r)], check=True, capture_output=True, text=True).stdout
        d = {}
        for line in out.splitlines():
            parts = line.split()
            if parts[0] == "dims":
                d["dims"] = [int(x) for x in parts[1:]]
            else:
                d[parts[0]] = np.array([float(x) for x in parts[2:]])
        return d
    return run


@pytest.mark.parametrize("p", [1, 2])
def test_tet_tables_equal_the_oracles(probe, p):
    T = probe("tet", p, 1)
    nv, nf, N, Nf, Nv, Q, dim = T["dims"]
    assert (nv, nf, N, Nf, Nv, Q, dim) == (p + 2, p + 1, 4 if p == 1 else 10, 3 if p == 1 else 6, 4, (p + 2) ** 3, 3)
    pts, wq = simplex3.volume_rule(nv)
    x, y, z = pts[:, 0], pts[:, 1], pts[:, 2]
    B = np.stack(simplex3.basis_values(p, x, y, z), axis=1)
    dB = np.stack([np.stack(g, axis=-1) for g in simplex3.basis_grads(p, x, y, z)], axis=1)
    V = np.stack(simplex3.basis_values(1, x, y, z), axis=1)
    dV = np.stack([np.stack(g, axis=-1) for g in simplex3.basis_grads(1, x, y, z)], axis=1)
    # the same closed forms in the same operation order: equal to the last bit
    assert np.array_equal(T["wq"], wq)
    assert np.array_equal(T["B"], B.ravel()) and np.array_equal(T["dB"], dB.ravel())
    assert np.array_equal(T["V"], V.ravel()) and np.array_equal(T["dV"], dV.ravel())
    t, w = gauss_legendre(nf)
    assert np.allclose(T["glf_t"], t, rtol=0, atol=1e-15) and np.allclose(T["glf_w"], w, rtol=0, atol=1e-15)


@pytest.mark.parametrize("p,r", [(1, 1), (2, 2), (3, 3), (2, 3)])
def test_triangle_tables_equal_the_oracles(probe, p, r):
    T = probe("tri", p, r)
    nv, nf, N, Nf, Nv, Q, dim = T["dims"]
    assert (N, Nf, Nv, dim) == ((p + 1) * (p + 2) // 2, p + 1, (r + 1) * (r + 2) // 2, 2)
    pts, wq = simplex.volume_rule(nv)
    dg = simplex.LagrangeTri(p, simplex.node_coords(p, gll_nodes(p)))
    geo = simplex.LagrangeTri(r, simplex.node_coords(r, equispaced_nodes(r)))
    assert Q == len(wq) and np.allclose(T["wq"], wq, rtol=0, atol=1e-15)
    # each side builds its Lagrange bases through its own Vandermonde inverse
    assert np.allclose(T["B"], dg.values(pts).ravel(), rtol=0, atol=1e-11)
    assert np.allclose(T["dB"], dg.grads(pts).ravel(), rtol=0, atol=1e-10)
    assert np.allclose(T["V"], geo.values(pts).ravel(), rtol=0, atol=1e-11)
    assert np.allclose(T["dV"], geo.grads(pts).ravel(), rtol=0, atol=1e-10)


@pytest.mark.parametrize("dim,p,r", [(2, 1, 2), (2, 3, 3), (3, 2, 2), (3, 1, 1)])
def test_tensor_tables_equal_the_oracles(probe, dim, p, r):
    from oracle.dg import n_vol_points
    from oracle.geometry import local_index_tuples, tensor_value
    T = probe(f"tensor{dim}", p, r)
    nv = T["dims"][0]
    assert nv == n_vol_points(p, r, dim)
    t, wt = gauss_legendre(nv)
    assert np.allclose(T["glv_t"], t, rtol=0, atol=1e-15) and np.allclose(T["glv_w"], wt, rtol=0, atol=1e-15)
    Q = nv ** dim
    idx = [[(q // nv ** k) % nv for k in range(dim)] for q in range(Q)]
    coords = [np.array([t[i[k]] for i in idx]) for k in range(dim)]
    gll = gll_nodes(p)
    tup = local_index_tuples(p, dim)
    B = np.stack([tensor_value(gll, tup[m], coords) * np.ones(Q) for m in range(len(tup))], 1)
    assert np.allclose(T["B"], B.ravel(), rtol=0, atol=1e-13)


@pytest.fixture(scope="module")
def tet_maps(tmp_path_factory):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("maps") / "tet_maps_probe")
    subprocess.run([nvcc, "-std=c++17", "-I", os.path.join(ROOT, "include"), "-gencode",
                    "arch=compute_103a,code=sm_103a", os.path.join(ROOT, "tests", "native", "tet_maps_probe.cu"),
                    "-o", exe], check=True, capture_output=True, text=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    faces, words, trace = {}, {}, {}
    for line in out.splitlines():
        k = line.split()
        if k[0] == "face":
            faces[(int(k[1]), int(k[2]))] = [int(x) for x in k[3:]]
        elif k[0] == "faceword":
            words[(int(k[1]), int(k[2]))] = int(k[3])
        else:
            trace[(int(k[1]), int(k[2]))] = int(k[3])
    return faces, words, trace


def test_tet_node_maps_of_the_sweep_kernels_equal_the_oracles(tet_maps):
    """Face nodes, the packed face-node words and the packed trace words of the TetEl policy,
    against the oracle's face_nodes and orientation permutations: our face node j of face f is
    the neighbour's face node seen through its face fn with code oc (vertices permuted by
    PERMS[oc], the midpoint of our face edge (j, j+1) the neighbour's midpoint of the permuted
    edge)."""
    faces, words, trace = tet_maps
    fe = {frozenset((0, 1)): 0, frozenset((1, 2)): 1, frozenset((2, 0)): 2}
    for p in (1, 2):
        NF, N = (3, 4) if p == 1 else (6, 10)
        for f in range(4):
            assert faces[(p, f)] == simplex3.face_nodes(p, f)
            for i in range(N):
                v = (words[(p, f)] >> (4 * i)) & 15
                fn_ = simplex3.face_nodes(p, f)
                assert v == (fn_.index(i) if i in fn_ else 15)
        for fn in range(4):
            for oc in range(6):
                w = trace[(p, fn * 6 + oc)]
                for j in range(NF):
                    pm = simplex3.PERMS[oc]
                    jn = pm[j] if j < 3 else 3 + fe[frozenset((pm[j - 3], pm[(j - 2) % 3]))]
                    assert (w >> (4 * j)) & 15 == simplex3.face_nodes(p, fn)[jn]
