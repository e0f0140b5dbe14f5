"""The library's representation-noise measurement (Sec. 4.B) on the GPU equals
the oracle's measurement on the CPU: same seeded inputs, same arithmetic
order, so the s(R_max, W) values agree exactly."""
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("dtype,form,W,ts", [
    ("f32", "sym", 2, range(48, 76, 3)),
    ("f32", "asym", 2, range(48, 76, 3)),
    ("f64", "sym", 3, range(64, 100, 4)),
    ("f64", "asym", 4, range(44, 80, 4)),
])
def test_gpu_calibration_equals_oracle(orc, dtype, form, W, ts):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1110_5765_gb300 import build
    build.build()
    from paper_1110_5765_gb300 import calibrate as gcal
    from oracle import calibrate as ocal
    got = gcal.calibrate_one(dtype, form, W, 128, ts=list(ts))
    ref = ocal.calibrate_one(dtype, form, W, 128, ts=list(ts))
    for t in ts:
        g, r = got[str(t)], ref[str(t)]
        assert (g["R"], g["q"], g["gA"], g["gB"]) == (r["R"], r["q"], r["gA"], r["gB"])
        assert g["s"] == r["s"] and g["m"] == r["m"], t
