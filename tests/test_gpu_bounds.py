"""The bounds-check mode: the library built with -DMCP_CHECK_BOUNDS (every
batch-array access of the persistent kernels tests its index; one out of
range is skipped and its source line recorded, nothing traps) runs small,
ragged cases of the thread, pair, group and segment kernels, records no
out-of-range access, and returns the normal build's results bit for bit (the
checks change no arithmetic)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2604_13323_gb300 import workloads as W  # noqa: E402
from tests.gpu_util import f32_exact  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def libs():
    from paper_2604_13323_gb300 import build, mcproj
    build.build()
    checked = mcproj.load_library(build.build_checked())
    return mcproj, mcproj.load_library(), checked


def _pair(mcproj, lib, chk, wl, **kw):
    a = mcproj.Projector(wl.robot, wl.constraints, wl.obstacles, lib=lib)
    b = mcproj.Projector(wl.robot, wl.constraints, wl.obstacles, lib=chk)
    assert a.bounds_status() == (0, 0) and b.bounds_status()[0] == 1
    return a, b


@pytest.mark.parametrize("name,n,ld", [("arm", 37, 64), ("arm", 4099, 4128), ("dual", 1001, 1024),
                                       ("humanoid", 259, 288)])
def test_checked_build_records_nothing_and_matches(libs, name, n, ld):
    mcproj, lib, chk = libs
    wl = {"arm": W.arm_workload(n=n), "dual": W.dual_arm_workload(total=10, n_random=n),
          "humanoid": W.humanoid_workload(n=n)}[name]
    a, b = _pair(mcproj, lib, chk, wl)
    q = torch.zeros((wl.dof, ld), dtype=torch.float32, device="cuda")
    q[:, :n] = torch.tensor(f32_exact(wl.q[:, :n]), dtype=torch.float32, device="cuda")
    if name == "dual":
        a.set_tuning(128, 4, 32, 0, 2)    # the pair kernel (one lane per arm)
        b.set_tuning(128, 4, 32, 0, 2)
    ra = a.project_check(q, wl.params, n=n)
    rb = b.project_check(q, wl.params, n=n)
    torch.cuda.synchronize()
    for x, y in zip(ra, rb):
        assert torch.equal(x[..., :n], y[..., :n])
    assert b.bounds_status(reset=True) == (1, 0)


def test_checked_build_segments(libs):
    mcproj, lib, chk = libs
    wl = W.dual_arm_workload(total=3000)
    ex = wl.extra
    a, b = _pair(mcproj, lib, chk, wl)
    starts = a.project(torch.tensor(ex["raw_start"], dtype=torch.float32, device="cuda"), wl.params)[0]
    delta = torch.tensor(ex["raw_dir"] * ex["step"], dtype=torch.float32, device="cuda")
    length = torch.tensor(ex["lengths"], dtype=torch.int32, device="cuda")
    ra = a.project_segments(starts, delta, length, wl.params)
    rb = b.project_segments(starts, delta, length, wl.params)
    torch.cuda.synchronize()
    for x, y in zip(ra, rb):
        assert torch.equal(x, y)
    assert b.bounds_status(reset=True) == (1, 0)
