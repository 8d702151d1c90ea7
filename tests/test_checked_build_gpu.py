"""The index-checked build (-DSVDLUT_CHECK_BOUNDS): every shared-memory
gather of the transform kernels is tested against its table size.  Over
edge-case sizes and dims the checked library must report no out-of-range
index and still match the FP64 oracle."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = r'''
import numpy as np, torch
import svdlut_inputs as si
import oracle
import paper_2508_16121_gb300 as sv
worst = 0.0
for (B, H, W, d) in [(1, 1, 1, si.spatial_dims(1, 1)), (1, 37, 130, si.spatial_dims(37, 130)),
                     (2, 67, 257, si.paper_dims()), (1, 70, 260, si.Dims(33, 33, 48, 9, 7, 64)),
                     (1, 45, 140, si.Dims(2, 1, 3, 2, 2, 2)), (1, 300, 515, si.Dims(17, 8, 8, 9, 5, 33))]:
    x, p = si.make_batch(5 + H, B, H, W, d)
    pd = sv.to_device(p)
    y = sv.apply(torch.from_numpy(x).cuda(), pd).cpu().numpy()
    worst = max(worst, float(np.abs(y - oracle.forward(d, p, x)).max()))
    dy = si.make_upstream(6 + H, x.shape)
    g = sv.backward(torch.from_numpy(x).cuda(), pd, torch.from_numpy(dy).cuda())
    torch.cuda.synchronize()
# pixel formats: interleaved 8-bit and 16-bit inputs (decoded to FP32 by
# their own kernel), ragged and 4-aligned widths
for (H, W) in [(37, 130), (64, 128), (2160, 3840)]:
    d = si.spatial_dims(H, W)
    x, p = si.make_batch(7 + H, 1, H, W, d)
    pd = sv.to_device(p)
    h8 = torch.from_numpy(si.to_hwc(si.to_u8(x))).cuda()
    v16 = np.stack([si.make_image_u16(np.random.default_rng(8 + H), H, W)])
    for _ in range(3):
        sv.apply_io(h8, pd, "u8_hwc", "u8_hwc")
        sv.apply_io(torch.from_numpy(v16).cuda(), pd, "u16", "u8")
        sv.apply_io(torch.from_numpy(si.to_hwc(v16)).cuda(), pd, "u16_hwc", "u8_hwc")
    torch.cuda.synchronize()
items = si.make_ragged(seed=9, n=3, sizes=((640, 480), (130, 37), (1, 1)))
ys = sv.apply_batched([torch.from_numpy(x).cuda() for x, _, _ in items], [sv.to_device(p) for _, _, p in items])
torch.cuda.synchronize()
rep = sv.check_report()
print("REPORT", rep, "WORST", worst)
assert rep is not None and rep["failures"] == 0, rep
assert worst <= 2e-5, worst
'''


def test_checked_build_reports_no_out_of_range_index(tmp_path):
    from paper_2508_16121_gb300 import build
    lib = str(tmp_path / "libsvdlut_checked.so")
    build.build(force=True, extra_flags=("-DSVDLUT_CHECK_BOUNDS",), out=lib)
    env = dict(os.environ, SVDLUT_LIB=lib)
    r = subprocess.run([sys.executable, "-c", CASES], cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    print(r.stdout[-2000:], r.stderr[-4000:])
    assert r.returncode == 0
    assert "REPORT" in r.stdout
