"""The library's host factorisation of the scalar elastic matrix (factor.cpp), compiled on its own
with g++ and checked on the CPU against its definition: with the nested-dissection permutation P,
S = L^{-1} must satisfy S (P A P^T) S^T = I; S is lower triangular; column j of S is stored on
exactly the elimination-tree path from j to its root; the ordering is a postorder of that tree, so
row i of S is the contiguous range of i's subtree; S^T is stored consistently; an indefinite
matrix is rejected.  Matrices: the oracle's elastic matrices of the cube and of a small beam,
and a random SPD matrix on a graph with two components."""
import os
import shutil
import subprocess

import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle.model import Mesh, elastic_matrix, lame

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA_INC = "/usr/local/cuda/include"


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path_factory.mktemp("factor") / "factor_harness")
    subprocess.run([cxx, "-std=c++17", "-O2", "-pthread", "-I", CUDA_INC,
                    os.path.join(ROOT, "paper_2603_16478_gb300", "csrc", "factor.cpp"),
                    os.path.join(ROOT, "tests", "factor_harness.cpp"), "-o", exe], check=True)
    return exe


def _run(harness, tmp_path, A, xyz):
    A = sp.csr_matrix(A)
    A.sort_indices()
    n = A.shape[0]
    src, dst = tmp_path / "in.bin", tmp_path / "out.bin"
    with open(src, "wb") as f:
        np.array([n], np.int32).tofile(f)
        np.array([A.nnz], np.int64).tofile(f)
        A.indptr.astype(np.int64).tofile(f)
        A.indices.astype(np.int32).tofile(f)
        A.data.astype(np.float64).tofile(f)
        np.ascontiguousarray(xyz, np.float64).tofile(f)
    r = subprocess.run([harness, str(src), str(dst)], capture_output=True, text=True)
    if r.returncode == 3:
        return r.stdout.strip()
    assert r.returncode == 0, r
    buf = open(dst, "rb").read()
    off = 0

    def take(dt, count):
        nonlocal off
        a = np.frombuffer(buf, dt, count, off)
        off += a.nbytes
        return a

    n_ = int(take(np.int32, 1)[0])
    nnz_L = int(take(np.int64, 1)[0])
    perm = take(np.int32, n_)
    parent = take(np.int32, n_)

    def csr():
        ptr = take(np.int64, n_ + 1)
        col = take(np.int32, int(ptr[-1]))
        val = take(np.float64, int(ptr[-1]))
        return sp.csr_matrix((val, col, ptr), shape=(n_, n_))

    S, St = csr(), csr()
    return dict(n=n_, nnz_L=nnz_L, perm=perm, parent=parent, S=S, St=St)


def _check(F, A):
    n = F["n"]
    perm = F["perm"]
    assert sorted(perm.tolist()) == list(range(n))
    Ap = sp.csr_matrix(A)[perm][:, perm]
    S = F["S"]
    assert sp.triu(S, 1).nnz == 0
    I = (S @ Ap @ S.T).toarray()
    assert np.abs(I - np.eye(n)).max() < 1e-10
    assert abs(F["St"] - S.T).max() == 0.0
    parent = F["parent"]
    assert all(parent[j] == -1 or parent[j] > j for j in range(n))
    St = F["St"]
    for j in range(n):
        path = []
        i = j
        while i != -1:
            path.append(i)
            i = parent[i]
        assert St.indices[St.indptr[j]:St.indptr[j + 1]].tolist() == path
    # the ordering is a postorder of the tree: every subtree is the contiguous range ending at its
    # root, so row i of S (the descendants of i) is exactly [i - size(i) + 1, i]
    size = np.ones(n, int)
    for j in range(n):
        if parent[j] >= 0:
            size[parent[j]] += size[j]
    for i in range(n):
        assert S.indices[S.indptr[i]:S.indptr[i + 1]].tolist() == list(range(i - size[i] + 1, i + 1))
    # nnz(L) counts the factor's nonzero pattern: L = S^{-1} has no entry outside it
    L = np.linalg.inv(S.toarray())
    assert np.count_nonzero(np.abs(np.tril(L)) > 1e-13 * np.abs(L).max()) <= F["nnz_L"]


def _scalar_elastic(pb):
    sc = pb.scene
    mesh = Mesh(sc.X, sc.tets)
    mu, _ = lame(sc.E, sc.nu)
    A3 = elastic_matrix(mesh, mesh.lumped_mass(sc.density), mu, sc.h).tocsr()
    As = A3[0::3, 0::3]
    assert abs(A3[1::3, 1::3] - As).max() <= 1e-14 * abs(As).max()  # A = A_s (x) I_3 up to summation order
    return As, sc.X


@pytest.mark.parametrize("name", ["cube", "beam"])
def test_factor_of_the_elastic_matrix(harness, tmp_path, name):
    pb = synth.cube_drop() if name == "cube" else synth.beam_incline(nx=12, ny=4, nz=3)
    As, X = _scalar_elastic(pb)
    F = _run(harness, tmp_path, As, X)
    _check(F, As)


def test_factor_of_a_graph_with_two_components(harness, tmp_path):
    rng = np.random.default_rng(3)
    n = 300
    xyz = rng.uniform(size=(n, 3))
    xyz[150:, 0] += 5.0  # two clouds
    rows, cols = [], []
    for i in range(n):
        lo, hi = (0, 150) if i < 150 else (150, n)
        for j in rng.choice(np.arange(lo, hi), 6, replace=False):
            if j != i:
                rows += [i, j]
                cols += [j, i]
    W = sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(n, n))
    W.data[:] = rng.uniform(0.5, 2.0, W.nnz)
    W = (W + W.T) * 0.5
    A = sp.diags(np.asarray(W.sum(axis=1)).ravel() + 0.1) - W
    F = _run(harness, tmp_path, A, xyz)
    _check(F, A)
    assert (F["parent"] == -1).sum() >= 2


def test_indefinite_matrix_is_rejected(harness, tmp_path):
    pb = synth.cube_drop()
    As, X = _scalar_elastic(pb)
    As = As.tolil()
    As[7, 7] = -1.0
    msg = _run(harness, tmp_path, As.tocsr(), X)
    assert isinstance(msg, str) and "positive definite" in msg


def test_parallel_factor_is_bit_identical_across_runs(harness, tmp_path):
    """Subtrees are factored by several threads in whatever order they finish; the result must
    not depend on it (each row sees exactly the data of a serial sweep)."""
    As, X = _scalar_elastic(synth.beam_incline(nx=16, ny=5, nz=4))
    runs = [_run(harness, tmp_path, As, X) for _ in range(4)]
    for F in runs[1:]:
        assert np.array_equal(F["perm"], runs[0]["perm"]) and np.array_equal(F["parent"], runs[0]["parent"])
        assert np.array_equal(F["S"].indices, runs[0]["S"].indices)
        assert np.array_equal(F["S"].data, runs[0]["S"].data)
