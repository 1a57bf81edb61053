"""The allocation-free pair sum (ls_pairsum_noalloc) against the regular one.

It serves callers that cannot allocate device memory (plug-ins whose device
memory belongs to a host application's allocator or a fixed pool, real-time
loops that must stay out of the allocator): its scratch is a static device array.
Checked through the C ABI against ls_pairsum_dev on two calls in a row (the
shared scratch keeps the previous call's contents), within the FP64 pair-sum
tolerance of the other parity tests.  This file is collected last on purpose.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2608_17615_b300 as L
from lsinput.workloads import random_density, two_material


def test_noalloc_matches_pairsum_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    wl = two_material("tiny", k=8.0)
    n = wl.mesh.n_nodes
    op = L.Operator(L.Mesh(wl.mesh), wl.k, wl.m, use_precond=0, pairsum=1)
    xy = torch.from_numpy(np.ascontiguousarray(wl.mesh.nodes)).cuda()
    w = torch.from_numpy(np.ascontiguousarray(wl.mesh.weights)).cuda()
    for seed in (21, 22):
        f = torch.from_numpy(random_density(n, seed)).cuda()
        ref = torch.empty_like(f)
        op.pairsum_dev(f, ref)
        y = torch.full_like(f, complex(np.nan, np.nan))
        L.pairsum_noalloc(xy, w, f, wl.k, y)
        err = (torch.linalg.norm(y - ref) / torch.linalg.norm(ref)).item()
        assert err < 1e-13, err


def test_noalloc_rejects_oversize():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    xy = torch.zeros((4, 2), dtype=torch.float64, device="cuda")
    w = torch.zeros(4, dtype=torch.float64, device="cuda")
    f = torch.zeros(4, dtype=torch.complex128, device="cuda")
    with pytest.raises(L.LsError) as e:
        L._check(L._lib.ls_pairsum_noalloc(2_000_000, L._dptr(xy), L._dptr(w), L._dptr(f), 5.0, L._dptr(f), None))
    assert "capacity" in str(e.value)
