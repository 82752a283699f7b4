"""The precision form at 512x512x80: error of every output field against the
FP64 oracle (run on the FP32-rounded inputs), for FP32 storage with binary32
hdiff and vadv in its three column-arithmetic forms (double-float also with its
column state in 48 bits, GTB_STATE48).  Bound: 1e-5 max-norm
relative; all-binary32 vadv is reported, not bounded (ill-conditioned columns
defeat it).  The measured errors are written to $GTB_REPORT_DIR/precision.json
when that variable is set."""
import json
import os

import numpy as np
import pytest

from helpers import region, rel_err, worst_column

pytestmark = pytest.mark.gpu
NAMES = ("u_stage", "wcon", "u_pos", "utens", "utens_stage")


def test_precision_form_errors(orc):
    import torch
    from paper_2311_08322_b300 import build, gtb, inputs
    build.build()
    I, J, K = 512, 512, 80
    f32 = {k: v.astype(np.float32) for k, v in inputs.hdiff_vadv(I, J, K, seed=0).items()}
    f64 = {k: v.astype(np.float64) for k, v in f32.items()}
    o2, o1 = (2, 2, 0), (1, 1, 0)
    ref_h = region(orc.hdiff(f64["in"], f64["coeff"]), o2, (I, J, K))
    ref_v = region(orc.vadv(*[f64[n] for n in NAMES]), o1, (I, J, K))
    s_in, s_cf = gtb.storage_from(f32["in"], o2), gtb.storage_from(f32["coeff"], o2)
    s_h = gtb.storage_from(np.zeros_like(f32["coeff"]), o2)
    gtb.hdiff(s_in, s_cf, s_h)
    st = {n: gtb.storage_from(f32[n], o1) for n in NAMES}
    report = {"workload": "512x512x80, FP32 storage, oracle in FP64 on the FP32-rounded inputs",
              "hdiff_fp32": {"max_norm_rel": rel_err(region(s_h.numpy(), o2, (I, J, K)), ref_h),
                             "worst_column": worst_column(region(s_h.numpy(), o2, (I, J, K)), ref_h)}}
    for prec, s48 in (("native", False), ("f64", False), ("df", False), ("df", True)):
        out = gtb.storage_from(np.zeros_like(f32["utens"]), o1)
        gtb.vadv(*[st[n] for n in NAMES], out, prec=prec, state48=s48)
        gtb.device_status()
        got = region(out.numpy(), o1, (I, J, K))
        report[f"vadv_fp32_{prec}{'48' if s48 else ''}"] = {"max_norm_rel": rel_err(got, ref_v),
                                                             "worst_column": worst_column(got, ref_v)}
    if os.environ.get("GTB_REPORT_DIR"):
        with open(os.path.join(os.environ["GTB_REPORT_DIR"], "precision.json"), "w") as fh:
            json.dump(report, fh, indent=1)
    print(json.dumps(report))
    assert report["hdiff_fp32"]["max_norm_rel"] <= 1e-5
    assert report["vadv_fp32_f64"]["max_norm_rel"] <= 1e-5
    assert report["vadv_fp32_df"]["max_norm_rel"] <= 1e-5
    assert report["vadv_fp32_df48"]["max_norm_rel"] <= 1e-5
