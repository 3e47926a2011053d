"""The allocation-free octree build (pse_build_octree_leaves_noalloc).

Callers that cannot allocate device memory -- plugins whose host application owns the
device allocator, real-time loops that must not wait on the allocator -- use this entry
point: its scratch is a fixed
file-scope device array and the leaf list goes into a buffer the caller owns.  It
must give exactly the leaves of pse_build_octree_from_tet_sizes, call after call
(the scratch keeps the previous call's contents, so it has to be cleared every time),
and it must refuse trees deeper than its fixed scratch can hold.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1612_09491_gb300 as pse  # noqa: E402
from paper_1612_09491_gb300 import _lib, build  # noqa: E402
from pse_inputs import lattice_positions, zeldovich_positions  # noqa: E402

pytestmark = pytest.mark.gpu


def squeezed_lattice(n, center, factor=0.3, radius=0.22, seed=0):
    q = lattice_positions(n).astype(np.float64)
    c = np.asarray(center)
    d = q - c
    r = np.linalg.norm(d, axis=1, keepdims=True)
    p = np.where(r < radius, c + d * factor, q)
    p = p + np.random.default_rng(seed).normal(0, 0.2 / n, p.shape)
    return np.mod(p, 1.0).astype(np.float32)


def noalloc_leaves(L, pos, n, bc, max_level, cap=8 ** 4, threshold=2.0, whole=True):
    dpos = torch.from_numpy(pos).cuda()
    lat = pse.lattice(n)
    d_leaves = torch.full((cap, 4), -1, dtype=torch.int32, device="cuda")
    d_n = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = L.pse_build_octree_leaves_noalloc(ctypes.c_void_p(dpos.data_ptr()), ctypes.byref(lat), bc, max_level,
                                           float(threshold), ctypes.c_void_p(d_leaves.data_ptr()), cap,
                                           ctypes.c_void_p(d_n.data_ptr()), stream)
    assert rc == _lib.PSE_OK, L.pse_last_error().decode()
    torch.cuda.synchronize()
    count = int(d_n.item())
    if not whole:
        return count, d_leaves.cpu().numpy()
    assert 0 < count <= cap
    return d_leaves[:count].cpu().numpy()


@pytest.fixture(scope="module")
def L():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    build.build()
    return _lib.load()


def test_noalloc_build_matches_allocating_build_on_consecutive_calls(L):
    n, bc, ml = 16, 4, 4
    inputs = [squeezed_lattice(n, (0.3, 0.6, 0.4), seed=1), squeezed_lattice(n, (0.7, 0.2, 0.5), seed=2),
              zeldovich_positions(n, -2.0, 1.0, seed=3)]
    for pos in inputs:  # consecutive calls share the scratch array
        got = noalloc_leaves(L, pos, n, bc, ml)
        exp = pse.build_octree_from_tet_sizes(torch.from_numpy(pos).cuda(), n, bc, ml, 2.0).leaves()
        np.testing.assert_array_equal(got, exp)


def test_noalloc_build_rejects_trees_beyond_its_scratch(L):
    pos = torch.from_numpy(lattice_positions(8)).cuda()
    lat = pse.lattice(8)
    d_leaves = torch.empty((16, 4), dtype=torch.int32, device="cuda")
    d_n = torch.empty((1,), dtype=torch.int64, device="cuda")
    rc = L.pse_build_octree_leaves_noalloc(ctypes.c_void_p(pos.data_ptr()), ctypes.byref(lat), 4, 5, 2.0,
                                           ctypes.c_void_p(d_leaves.data_ptr()), 16,
                                           ctypes.c_void_p(d_n.data_ptr()), None)
    assert rc == _lib.PSE_ERR_INVALID_ARG
    assert "scratch" in L.pse_last_error().decode()


def test_noalloc_build_thresholds_on_bin_edges(L):
    """A threshold equal to a histogram bin's lower edge: the cutoff is taken on the host the
    way the allocating build compares edges, so both give the same leaves."""
    n, bc, ml = 16, 4, 4
    pos = squeezed_lattice(n, (0.4, 0.4, 0.6), seed=7)
    for b in (28, 30, 33, 36):
        thr = 10.0 ** (-3.0 + 6.0 * b / 64.0)
        got = noalloc_leaves(L, pos, n, bc, ml, threshold=thr)
        exp = pse.build_octree_from_tet_sizes(torch.from_numpy(pos).cuda(), n, bc, ml, thr).leaves()
        np.testing.assert_array_equal(got, exp)


def test_noalloc_build_truncates_at_cap_and_builds_one_level(L):
    n, bc, ml = 16, 4, 4
    pos = squeezed_lattice(n, (0.3, 0.6, 0.4), seed=1)
    exp = pse.build_octree_from_tet_sizes(torch.from_numpy(pos).cuda(), n, bc, ml, 2.0).leaves()
    assert len(exp) > 8
    cap = len(exp) // 2
    count, buf = noalloc_leaves(L, pos, n, bc, ml, cap=cap, whole=False)
    assert count == len(exp)                       # the full count, so the caller can retry
    np.testing.assert_array_equal(buf, exp[:cap])  # and the first cap leaves
    root = noalloc_leaves(L, pos, n, bc, 0)        # max_level 0: the root alone
    np.testing.assert_array_equal(root, [[0, 0, 0, 0]])


def test_noalloc_build_captured_in_a_graph_and_replayed(L):
    """The stated use: after one call outside capture (which resolves the scratch array's
    address), the call is captured in a CUDA graph and replayed; each replay writes the
    leaves of the allocating build for the positions the graph reads at that moment."""
    n, bc, ml = 16, 4, 4
    pos_a = squeezed_lattice(n, (0.3, 0.6, 0.4), seed=1)
    pos_b = squeezed_lattice(n, (0.7, 0.2, 0.5), seed=2)
    exp_a = pse.build_octree_from_tet_sizes(torch.from_numpy(pos_a).cuda(), n, bc, ml, 2.0).leaves()
    exp_b = pse.build_octree_from_tet_sizes(torch.from_numpy(pos_b).cuda(), n, bc, ml, 2.0).leaves()
    noalloc_leaves(L, pos_a, n, bc, ml)  # first call, outside capture
    dpos = torch.from_numpy(pos_a).cuda()
    lat = pse.lattice(n)
    cap = 8 ** 4
    d_leaves = torch.full((cap, 4), -1, dtype=torch.int32, device="cuda")
    d_n = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        with torch.cuda.graph(graph, stream=side):
            rc = L.pse_build_octree_leaves_noalloc(ctypes.c_void_p(dpos.data_ptr()), ctypes.byref(lat), bc, ml, 2.0,
                                                   ctypes.c_void_p(d_leaves.data_ptr()), cap,
                                                   ctypes.c_void_p(d_n.data_ptr()), ctypes.c_void_p(side.cuda_stream))
    assert rc == _lib.PSE_OK, L.pse_last_error().decode()
    torch.cuda.current_stream().wait_stream(side)
    for pos, exp in ((pos_a, exp_a), (pos_b, exp_b)):
        dpos.copy_(torch.from_numpy(pos))
        d_leaves.fill_(-1)
        graph.replay()
        torch.cuda.synchronize()
        count = int(d_n.item())
        assert count == len(exp)
        np.testing.assert_array_equal(d_leaves[:count].cpu().numpy(), exp)
