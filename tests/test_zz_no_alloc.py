"""rpba_sigma0_noalloc: sigma_0 and RMS without any device allocation.

Callers that cannot allocate device memory per call (a fixed device-memory
budget, an allocator owned by another framework) use this entry point; its
only scratch is one fixed array in the library. The test gives it a block that
lives in device memory the caller owns and checks its result against the
context-based rpba_sigma0 on the same state, on two calls in a row (the shared
scratch keeps the previous call's contents, so the second call must not
depend on them).
"""

import numpy as np
import pytest

from paper_1910_08138_gb300 import rpba, synth

pytestmark = pytest.mark.gpu

MAX_OBS = 8192 * 256  # RPBA_NOALLOC_MAX_OBS of include/rpba.h


def test_sigma0_noalloc_matches_context_entry_point_twice():
    import torch
    from scipy.spatial.transform import Rotation

    prob = synth.config(1)
    g = rpba.Rpba(prob, robust=1, robust_from_start=1)
    g.iterate(2)  # robust weights and eliminated points make the state non-trivial
    s_ref, rms_ref = g.sigma0()
    pose = g.cameras()
    X, act = g.points()
    w = g.weights()
    assert (act == 0).any() and (w != 1.0).any()

    dev = torch.device("cuda")
    f64 = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    i32 = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.int32, device=dev)
    R = f64(Rotation.from_rotvec(pose[:, :3]).as_matrix().reshape(-1, 9))
    t = f64(pose[:, 3:])
    intr = f64(prob["cam_intr"])
    Xd = f64(X)
    actd = torch.tensor(act, dtype=torch.uint8, device=dev)
    oc, op, xy, wd = i32(prob["obs_cam"]), i32(prob["obs_point"]), f64(prob["obs_xy"]), f64(w)
    stream = torch.cuda.current_stream()
    results = []
    for _ in range(2):
        s0, rms, sums = rpba.rpba_sigma0_noalloc(
            g.M, g.N, g.K, R.data_ptr(), t.data_ptr(), intr.data_ptr(), Xd.data_ptr(), actd.data_ptr(),
            oc.data_ptr(), op.data_ptr(), xy.data_ptr(), None, wd.data_ptr(), stream=stream)
        assert s0 == pytest.approx(s_ref, rel=1e-10)
        assert rms == pytest.approx(rms_ref, rel=1e-10)
        assert sums[4] == act.sum()
        results.append((s0, rms))
    assert results[0] == results[1]


def test_sigma0_noalloc_rejects_blocks_above_its_limit():
    with pytest.raises(rpba.RpbaError) as e:
        rpba.rpba_sigma0_noalloc(1, 1, MAX_OBS + 1, 1, 1, 1, 1, None, 1, 1, 1)
    assert e.value.status == 1  # RPBA_ERR_INVALID_ARG, nothing launched
    # observations that reference no camera or no point: rejected on the host.
    # Every array is a real device buffer large enough for one camera, point
    # and observation, so no launch could read outside memory it owns.
    import torch
    dev = torch.device("cuda")
    buf = torch.zeros(64, dtype=torch.float64, device=dev)
    idx = torch.zeros(4, dtype=torch.int32, device=dev)
    for n_cams, n_points in ((0, 1), (1, 0)):
        with pytest.raises(rpba.RpbaError) as e:
            rpba.rpba_sigma0_noalloc(n_cams, n_points, 1, buf.data_ptr(), buf.data_ptr(), buf.data_ptr(),
                                     buf.data_ptr(), None, idx.data_ptr(), idx.data_ptr(), buf.data_ptr())
        assert e.value.status == 1
