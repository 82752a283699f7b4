"""The checked build (libgtb_checked.so, loaded when GTB_CHECKED=1): the same kernels,
each testing the first and last element of every run of addresses it touches against
the storage the host declared for that field, and reporting a run outside it through
gtb_device_status instead of touching it.  compute-sanitizer is not available on
these GPUs; this build checks the kernels' index arithmetic in its place.

One battery of calls (every entry point, both storage types, every column arithmetic,
ragged shapes, storages padded on every side with the domain at an offset origin) runs
in a child process once with each library.  With the checked library every call must
leave the device status clean, and both libraries must produce the same storages bit
for bit, padding included."""
import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def battery(path):
    sys.path.insert(0, ROOT)
    import torch
    from paper_2311_08322_b300 import gtb, inputs

    checked = os.environ.get("GTB_CHECKED") == "1"
    assert ("checked" in gtb.version()) == checked, gtb.version()
    outs = {}
    pad = ((1, 2), (1, 3), (2, 5))  # k, j, i: the domain sits at an offset inside its storage

    def up(arr, halo, dt):
        a = np.pad(arr, pad, mode="constant", constant_values=7.25).astype(dt)
        return gtb.storage_from(a, (halo + pad[2][0], halo + pad[1][0], pad[0][0]))

    def zeros_like(st):
        return gtb.Storage(st.data.clone().fill_(-3.5), st.origin)

    def keep(tag, *sts):
        gtb.device_status()  # raises GtbError on a run outside a storage (checked build)
        for q, st in enumerate(sts):
            outs[f"{tag}.{q}"] = st.numpy()

    names = ("u_stage", "wcon", "u_pos", "utens", "utens_stage")
    for dt, I, J, K in ((np.float64, 67, 45, 7), (np.float32, 70, 33, 9)):
        f = inputs.hdiff_vadv(I, J, K, seed=5)
        dom = (I, J, K)
        tdt = torch.float64 if dt == np.float64 else torch.float32
        s_in, s_cf = up(f["in"], 2, dt), up(f["coeff"], 2, dt)
        s_h = zeros_like(s_cf)
        gtb.hdiff(s_in, s_cf, s_h, domain=dom)
        keep(f"hdiff.{dt.__name__}", s_h)
        sv = {n: up(f[n], 1, dt) for n in names}
        precs = ("native",) if dt == np.float64 else ("native", "f64", "df")
        for pr in precs:
            for literal, beta in ((False, 0.0), (True, 0.0), (False, 0.3)):
                o = zeros_like(sv["utens"])
                gtb.vadv(*[sv[n] for n in names], o, prec=pr, literal=literal, beta_v=beta, domain=dom)
                keep(f"vadv.{dt.__name__}.{pr}.{literal}.{beta}", o)
            if pr == "df":  # the column state in 48 bits
                o = zeros_like(sv["utens"])
                gtb.vadv(*[sv[n] for n in names], o, prec=pr, domain=dom, state48=True)
                keep(f"vadv_state48.{dt.__name__}", o)
                h2, o2 = zeros_like(s_cf), zeros_like(sv["utens"])
                gtb.step(s_in, s_cf, h2, *[sv[n] for n in names], o2, prec=pr, domain=dom, state48=True)
                keep(f"step_state48.{dt.__name__}", h2, o2)
            o = zeros_like(sv["utens"])
            gtb.vadv(*[sv[n] for n in names], o, prec=pr, domain=dom, workspace=None)  # shared-memory state
            keep(f"vadv_smem.{dt.__name__}.{pr}", o)
            ip = gtb.Storage(sv["utens_stage"].data.clone(), sv["utens_stage"].origin)  # in place
            gtb.vadv(sv["u_stage"], sv["wcon"], sv["u_pos"], sv["utens"], ip, prec=pr, domain=dom)
            keep(f"vadv_inplace.{dt.__name__}.{pr}", ip)
            h2, o2 = zeros_like(s_cf), zeros_like(sv["utens"])
            gtb.step(s_in, s_cf, h2, *[sv[n] for n in names], o2, prec=pr, domain=dom)
            keep(f"step.{dt.__name__}.{pr}", h2, o2)
            o3 = zeros_like(sv["utens"])
            gtb.hdiff_vadv(s_in, s_cf, sv["wcon"], sv["utens"], sv["utens_stage"], o3, prec=pr, domain=dom)
            keep(f"chain.{dt.__name__}.{pr}", o3)
            # kept factors, then the adjoint on them and the refactorising adjoint
            F = torch.empty(gtb.hdiff_vadv_workspace_bytes(tdt, pr, dom, save_factors=True), dtype=torch.uint8,
                            device="cuda")
            o4 = zeros_like(sv["utens"])
            gtb.hdiff_vadv(s_in, s_cf, sv["wcon"], sv["utens"], sv["utens_stage"], o4, prec=pr, domain=dom,
                           workspace=F, save_factors=True)
            keep(f"chain_factors.{dt.__name__}.{pr}", o4)
            a1, c1 = zeros_like(sv["utens"]), zeros_like(sv["utens"])
            gtb.vadv_adj(sv["wcon"], sv["u_pos"], a1, a1, c1, prec=pr, domain=dom, workspace=F, factors=True)
            a2, b2, c2, d2 = (zeros_like(sv["utens"]) for _ in range(4))
            gtb.vadv_adj(sv["wcon"], sv["u_pos"], a2, b2, c2, d2, prec=pr, domain=dom, beta_v=0.3)
            keep(f"vadv_adj.{dt.__name__}.{pr}", a1, c1, a2, b2, c2, d2)
        ib, cb = zeros_like(s_in), zeros_like(s_cf)
        gtb.hdiff_adj(s_in, s_cf, s_h, ib, cb, domain=dom)
        gtb.hdiff_adj(s_in, s_cf, s_cf, ib, cb, accumulate=True, domain=dom)
        keep(f"hdiff_adj.{dt.__name__}", ib, cb)
        hp = gtb.Storage(s_in.data.clone(), s_in.origin)
        gtb.halo_periodic(hp, domain=dom)
        keep(f"halo.{dt.__name__}", hp)
        gtb.halo_periodic_adj(hp, domain=dom)
        keep(f"halo_adj.{dt.__name__}", hp)
        # ensembles: three uneven members in one plan
        mems = []
        for q, (mi, mj, mk) in enumerate(((48, 40, 9), (66, 17, 5), (32, 50, 12))):
            fm = inputs.hdiff_vadv(mi, mj, mk, seed=20 + q)
            mems.append(gtb.member_storages({k: v.astype(dt) for k, v in fm.items()}, mi, mj, mk))
        plan = gtb.BatchPlan(mems, prec="df" if dt == np.float32 else "native")
        plan.run()
        keep(f"batch.{dt.__name__}", *[m["h"] for m in mems], *[m["out"] for m in mems])
        plan.close()
    # the allocation-free vadv (binary64)
    f = inputs.hdiff_vadv(40, 24, 6, seed=9)
    sv = {n: up(f[n], 1, np.float64) for n in names}
    o = zeros_like(sv["utens"])
    fs = [gtb.field(sv[n]) for n in names] + [gtb.field(o)]
    dom = (ctypes.c_int64 * 3)(40, 24, 6)
    rc = gtb.lib().gtb_vadv_noalloc(*[ctypes.byref(x) for x in fs], 0.15, 0.0, 0, 0, dom,
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, gtb.lib().gtb_last_error().decode()
    keep("vadv_noalloc", o)
    np.savez(path, **outs)
    print(f"{len(outs)} storages, {gtb.version()}")


@pytest.mark.gpu
def test_checked_build_is_clean_and_bit_identical(tmp_path):
    sys.path.insert(0, ROOT)
    from paper_2311_08322_b300 import build
    build.build()  # both libraries, if missing or older than the sources
    env_default = {k: v for k, v in os.environ.items() if k != "GTB_CHECKED"}
    env_checked = dict(env_default, GTB_CHECKED="1")
    for name, env in (("default", env_default), ("checked", env_checked)):
        r = subprocess.run([sys.executable, os.path.abspath(__file__), str(tmp_path / f"{name}.npz")], env=env,
                           capture_output=True, text=True, timeout=900)
        assert r.returncode == 0, f"{name}:\n{r.stdout}\n{r.stderr[-4000:]}"
        print(name, r.stdout.strip())
    a, b = np.load(tmp_path / "default.npz"), np.load(tmp_path / "checked.npz")
    assert sorted(a.files) == sorted(b.files)
    for k in a.files:
        assert np.array_equal(a[k], b[k], equal_nan=True), k


if __name__ == "__main__":
    battery(sys.argv[1])
