"""Device build of the VDIM correction dV against the host build.

The host build (long double, OpenMP) is pinned to the oracle on the CPU
(tests/test_lib_cpu.py, <= 1e-13 relative).  The device build evaluates the
same Green's-identity boundary moments and plain-quadrature patch moments in
double-double arithmetic on the GPU with the same work list (patches, panels)
and the same long-double coefficient matrices, so the two differ only by the
host's extended-precision rounding.  That rounding is measured by comparing two
independent long-double builds, the host's and the oracle's: they agree to
1.2e-13 of max |dV| on the two-material mesh and to < 1e-13 on the other two
(on a coarser 810-node disk with larger patches, where |E|/|dV| grows, they
differ by 3.8e-12).  The bar is twice that level, 2e-13 of max |dV|, entry by
entry, with identical sparsity; the device build itself carries about 30 digits.  Meshes: the constant disk (circular arcs), the
two-material disk (an interface: blocks of two subdomains per target) and a
star scatterer (arcs of r = 1 + 0.2 cos(5 t + phi), so the double-double sine
and cosine of the curve enter).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2608_17615_b300 as L
from lsinput.workloads import constant_disk, star_scatterer, two_material


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


CASES = {
    "disk": lambda: constant_disk(k=5.0, n_rings=2),
    "two_material": lambda: two_material("tiny", k=8.0),
    "star": lambda: star_scatterer(1, 3000, k=10.0),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_device_correction_matches_host(name):
    wl = CASES[name]()
    M = L.Mesh(wl.mesh)
    rp_h, ci_h, va_h = L.correction_host(M, wl.k, 3.0)
    rp_d, ci_d, va_d, nhost = L.correction_dev(M, wl.k, 3.0)
    assert np.array_equal(rp_h, rp_d) and np.array_equal(ci_h, ci_d)
    err = np.max(np.abs(va_d - va_h)) / np.max(np.abs(va_h))
    print(name, "device vs host dV", err, "host-rebuilt blocks", nhost)
    assert nhost == 0
    assert err < 2e-13


def test_operator_setup_on_device_matches_host_setup():
    # the two setups differ by the host build's rounding of dV (about 1e-13 of max |dV|
    # here), which reaches L x through k^2 dV m x; the bar stays 10x under the 1e-11
    # FP64 matvec bar against the oracle
    wl = two_material("tiny", k=8.0)
    M = L.Mesh(wl.mesh)
    x = torch.from_numpy(np.exp(1j * np.arange(wl.mesh.n_nodes) * 0.3)).cuda()
    ys = []
    for dev in (1, 0):
        op = L.Operator(M, wl.k, wl.m, use_precond=0, setup_on_device=dev)
        y = torch.empty_like(x)
        op.apply_dev(x, y)
        ys.append(y)
    assert (torch.linalg.norm(ys[0] - ys[1]) / torch.linalg.norm(ys[1])).item() < 1e-12
