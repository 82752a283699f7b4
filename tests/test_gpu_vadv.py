"""GPU parity of gtb_vadv against the FP64 oracle (GT4Py paper Sec. 3.1,
implicit vertical advection: FORWARD elimination then BACKWARD substitution).
FP64 bound: 1e-12 max-norm relative.  FP32 storage: the oracle runs in FP64 on
the FP32-rounded inputs; the FP64-arithmetic and double-float forms must stay
within 1e-5, the all-FP32 form is only reported (it cannot meet the bound on
ill-conditioned columns)."""
import numpy as np
import pytest

from helpers import region, rel_err, worst_column

pytestmark = pytest.mark.gpu

F64_TOL = 1e-12
F32_TOL = 1e-5
NAMES = ("u_stage", "wcon", "u_pos", "utens", "utens_stage")


@pytest.fixture(scope="module")
def G():
    import torch
    from paper_2311_08322_b300 import build, gtb
    assert torch.cuda.is_available()
    build.build()
    return gtb


def draw(I, J, K, seed, wamp=0.5, pad=(0, 0, 0)):
    rng = np.random.default_rng(seed)
    shp = (K + 2 * pad[2], J + 2 + 2 * pad[1], I + 2 + 2 * pad[0])
    f = {n: rng.uniform(-1, 1, shp) for n in ("u_stage", "u_pos", "utens", "utens_stage")}
    f["wcon"] = rng.uniform(-wamp, wamp, shp)
    return f


def run_case(G, orc, I, J, K, seed=0, dtype=np.float64, prec="native", pad=(0, 0, 0), inplace=False,
             literal=False, beta_v=0.0, wamp=0.5, f=None, workspace="auto"):
    f = draw(I, J, K, seed, wamp, pad) if f is None else f
    if dtype == np.float32:
        f = {k: v.astype(np.float32) for k, v in f.items()}
    o = (1 + pad[0], 1 + pad[1], pad[2])
    dom = (I, J, K)
    st = {n: G.storage_from(f[n], o) for n in NAMES}
    out = st["utens_stage"] if inplace else G.storage_from(np.zeros_like(f["utens_stage"]), o)
    G.vadv(*[st[n] for n in NAMES], out, prec=prec, literal=literal, beta_v=beta_v, domain=dom, workspace=workspace)
    G.device_status()
    got = region(out.numpy(), o, dom)
    ref = orc.vadv(*[f[n].astype(np.float64) for n in NAMES], origin=o, domain=dom, beta_v=beta_v,
                   wmode=1 if literal else 0)
    return got, region(ref, o, dom)


def test_256_fp64_full_field(G, orc):
    """256x256x80 FP64, wcon ~ U(-0.5,0.5), dtr_stage = 3/20, beta_v = 0; whole field."""
    got, ref = run_case(G, orc, 256, 256, 80, seed=0)
    e = rel_err(got, ref)
    assert e <= F64_TOL, (e, worst_column(got, ref))


@pytest.mark.parametrize("I,J,K", [(64, 64, 40), (33, 7, 1), (1, 1, 2), (31, 5, 3), (70, 9, 137), (3, 65, 17)])
def test_shapes_fp64(G, orc, I, J, K):
    """Ragged warps in I, odd J, and K = 1, 2, 3 (degenerate top/bottom intervals), 137."""
    got, ref = run_case(G, orc, I, J, K, seed=I * J + K)
    assert rel_err(got, ref) <= F64_TOL


def test_max_k_fp64(G, orc):
    """K = 448, the largest K whose column state fits shared memory."""
    got, ref = run_case(G, orc, 40, 3, 448, seed=9, wamp=0.15)
    assert rel_err(got, ref) <= F64_TOL


def test_k_beyond_limit_rejected(G):
    """Without a workspace the column state lives in shared memory: K <= 448."""
    f = draw(4, 2, 449, 1)
    st = {n: G.storage_from(f[n], (1, 1, 0)) for n in NAMES}
    with pytest.raises(G.GtbError) as e:
        G.vadv(*[st[n] for n in NAMES], G.storage_from(np.zeros_like(f["utens"]), (1, 1, 0)), workspace=None)
    assert e.value.code == -8


def test_large_k_with_workspace_fp64(G, orc):
    """With a workspace any K runs: K = 1000."""
    got, ref = run_case(G, orc, 33, 3, 1000, seed=10, wamp=0.15)
    assert rel_err(got, ref) <= F64_TOL


def test_in_place(G, orc):
    """utens_stage_out is the very same storage as utens_stage."""
    got, ref = run_case(G, orc, 100, 30, 60, seed=4, inplace=True)
    assert rel_err(got, ref) <= F64_TOL


@pytest.mark.parametrize("pad", [(1, 0, 0), (2, 3, 1)])
def test_origin_offsets(G, orc, pad):
    got, ref = run_case(G, orc, 45, 12, 20, seed=5, pad=pad)
    assert rel_err(got, ref) <= F64_TOL


def test_literal_wcon_and_beta(G, orc):
    """The literal face-velocity reading and a nonzero beta_v (both parity-unpinned
    readings) agree with the oracle's statement of them."""
    for literal, beta in ((True, 0.0), (False, 0.3), (True, -0.2)):
        got, ref = run_case(G, orc, 50, 11, 30, seed=6, literal=literal, beta_v=beta, wamp=0.3)
        assert rel_err(got, ref) <= F64_TOL, (literal, beta)


@pytest.mark.parametrize("prec,tol", [("f64", F32_TOL), ("df", F32_TOL)])
def test_fp32_storage_512(G, orc, prec, tol):
    """512x512x80 FP32 storage; FP64 or double-float column arithmetic meets 1e-5."""
    got, ref = run_case(G, orc, 512, 512, 80, seed=0, dtype=np.float32, prec=prec)
    e = rel_err(got, ref)
    assert e <= tol, (prec, e, worst_column(got, ref))


def test_fp32_native_reported(G, orc):
    """All-binary32 column arithmetic: finite, but its error on ill-conditioned columns
    is far above the FP32 bound (which is why the mixed forms exist)."""
    got, ref = run_case(G, orc, 128, 128, 80, seed=0, dtype=np.float32, prec="native")
    assert np.all(np.isfinite(got))
    assert rel_err(got, ref) < 1.0


@pytest.mark.parametrize("prec", ["native", "f64", "df"])
def test_fp32_ragged(G, orc, prec):
    got, ref = run_case(G, orc, 37, 6, 9, seed=8, dtype=np.float32, prec=prec, wamp=0.15)
    assert rel_err(got, ref) <= (F32_TOL if prec != "native" else 1e-4)


@pytest.mark.parametrize("literal,beta_v", [(False, 0.0), (True, 0.0), (False, 0.3)])
def test_df_column_pairs_equal_single_columns(G, literal, beta_v):
    """Double-float columns two per thread (binary32 storages whose column pairs are
    8-byte aligned, I even) give, bit for bit, what one column per thread gives: the same
    values in storages shifted by one element, whose pairs are not aligned."""
    import torch
    I, J, K = 130, 34, 45
    f = {k: v.astype(np.float32) for k, v in draw(I, J, K, seed=12, wamp=0.4).items()}
    o, dom = (1, 1, 0), (I, J, K)

    def storages(shift):
        st = {}
        for n in NAMES + ("out",):
            a = np.zeros_like(f["utens_stage"]) if n == "out" else f[n]
            nk, nj, ni = a.shape
            t = G.empty_storage(ni + 1, nj, nk, dtype=torch.float32, halo_i=o[0])
            v = t[:, :, 1:] if shift else t[:, :, :ni]
            v.copy_(torch.from_numpy(np.ascontiguousarray(a)))
            st[n] = G.Storage(v, o)
        return st

    outs = []
    for shift in (False, True):
        st = storages(shift)
        # domain column 0 8-byte aligned (pairs) only in the unshifted storages
        assert ((st["u_stage"].data.data_ptr() + 4 * o[0]) % 8 == 0) != shift
        G.vadv(*[st[n] for n in NAMES], st["out"], prec="df", literal=literal, beta_v=beta_v, domain=dom)
        G.device_status()
        outs.append(region(st["out"].numpy(), o, dom))
    assert np.array_equal(outs[0].view(np.uint32), outs[1].view(np.uint32))


def test_zero_pivot_column(G, orc):
    """b_0 = 0 exactly (dtr = 1/4, wcon = 1 on both faces of level 1): the unpivoted
    solve breaks down in that column on both sides; every other column is exact."""
    I, J, K = 8, 2, 5
    f = draw(I, J, K, 12, 0.1)
    f["wcon"][1, 1, 3:5] = 1.0  # column (i=2, j=0): w_1 = 1, c_0 = w_1/4 = dtr, so b_0 = 0
    o = (1, 1, 0)
    st = {n: G.storage_from(f[n], o) for n in NAMES}
    out = G.storage_from(np.zeros_like(f["utens"]), o)
    G.vadv(*[st[n] for n in NAMES], out, dtr_stage=0.25)
    G.device_status()
    got = region(out.numpy(), o, (I, J, K))
    ref = region(orc.vadv(*[f[n] for n in NAMES], dtr_stage=0.25), o, (I, J, K))
    bad_ref = ~np.all(np.isfinite(ref), axis=0)
    bad_got = ~np.all(np.isfinite(got), axis=0)
    assert bad_ref[0, 2] and np.array_equal(bad_ref, bad_got)
    assert rel_err(got[:, ~bad_ref], ref[:, ~bad_ref]) <= F64_TOL


@pytest.mark.parametrize("dtype,prec", [(np.float64, "native"), (np.float32, "df"), (np.float32, "f64"),
                                        (np.float32, "native")])
def test_shared_memory_form(G, orc, dtype, prec):
    """Without a workspace the column state stays in shared memory; same results."""
    tol = F64_TOL if dtype == np.float64 else (F32_TOL if prec != "native" else 1e-4)
    for I, J, K in ((256, 64, 80), (45, 7, 137), (33, 3, 1)):
        got, ref = run_case(G, orc, I, J, K, seed=K, dtype=dtype, prec=prec, wamp=0.15 if prec == "native" else 0.5,
                            workspace=None)
        assert rel_err(got, ref) <= tol, (I, J, K)


def test_explicit_workspace_tensor_and_inplace(G, orc):
    import torch
    need = G.vadv_workspace_bytes(torch.float64, "native", (60, 20, 50))
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    got, ref = run_case(G, orc, 60, 20, 50, seed=77, inplace=True, workspace=ws)
    assert rel_err(got, ref) <= F64_TOL


@pytest.mark.parametrize("workspace", ["auto", None])
@pytest.mark.parametrize("dtype,prec", [(np.float64, "native"), (np.float32, "df"), (np.float32, "f64")])
def test_general_weights_every_form(G, orc, workspace, dtype, prec):
    """beta_v != 0 (the general-weight body of the column solve) and the literal face
    velocity in every state form (workspace: the y back substitution in binary64, e_k
    otherwise; shared memory: e_k) and column arithmetic."""
    tol = F64_TOL if dtype == np.float64 else F32_TOL
    for literal, beta in ((False, 0.3), (True, -0.2), (True, 0.0)):
        got, ref = run_case(G, orc, 67, 13, 41, seed=9, dtype=dtype, prec=prec, literal=literal, beta_v=beta,
                            wamp=0.25, workspace=workspace)
        assert rel_err(got, ref) <= tol, (literal, beta)


@pytest.mark.parametrize("I,J,K,literal,beta_v,inplace", [
    (130, 34, 45, False, 0.0, False),  # column pairs, ragged J
    (129, 9, 37, False, 0.0, False),   # odd I: one column a thread
    (96, 40, 137, True, 0.0, True),    # literal face velocity, in place, the ensemble's largest K
    (70, 33, 41, False, 0.3, False),   # general weights
])
def test_state48_fp32_df(G, orc, I, J, K, literal, beta_v, inplace):
    """GTB_STATE48: double-float columns whose workspace state is kept in 48 bits meet the
    1e-5 bound against the FP64 oracle and differ from the full-width form in the last
    bits; without a workspace (shared-memory state) the flag has no effect, bit for bit."""
    f = {k: v.astype(np.float32) for k, v in draw(I, J, K, seed=17).items()}
    o, dom = (1, 1, 0), (I, J, K)
    ref = region(orc.vadv(*[f[n].astype(np.float64) for n in NAMES], origin=o, domain=dom, beta_v=beta_v,
                          wmode=1 if literal else 0), o, dom)
    outs = []
    for state48, ws in ((True, "auto"), (False, "auto"), (True, None), (False, None)):
        st = {n: G.storage_from(f[n], o) for n in NAMES}
        out = st["utens_stage"] if inplace else G.storage_from(np.zeros_like(f["utens_stage"]), o)
        G.vadv(*[st[n] for n in NAMES], out, prec="df", literal=literal, beta_v=beta_v, domain=dom, workspace=ws,
               state48=state48)
        G.device_status()
        outs.append(region(out.numpy(), o, dom))
    assert rel_err(outs[0], ref) <= F32_TOL
    assert rel_err(outs[1], ref) <= F32_TOL
    assert not np.array_equal(outs[0].view(np.uint32), outs[1].view(np.uint32))
    assert np.array_equal(outs[2].view(np.uint32), outs[3].view(np.uint32))


def test_state48_rejected_outside_df_fp32(G):
    f = draw(8, 8, 4, seed=1)
    for dt, prec in ((np.float64, "native"), (np.float32, "native"), (np.float32, "f64")):
        st = {n: G.storage_from(f[n].astype(dt), (1, 1, 0)) for n in NAMES}
        with pytest.raises(G.GtbError) as e:
            G.vadv(*[st[n] for n in NAMES], prec=prec, state48=True)
        assert e.value.code == -9


def test_state48_zero_pivot_column(G, orc):
    """GTB_STATE48 on the zero-pivot column of test_zero_pivot_column (binary32 storage,
    column pairs): the breakdown stays in that column, every other column meets 1e-5."""
    I, J, K = 8, 2, 5
    f = draw(I, J, K, 12, 0.1)
    f["wcon"][1, 1, 3:5] = 1.0
    f = {k: v.astype(np.float32) for k, v in f.items()}
    o = (1, 1, 0)
    st = {n: G.storage_from(f[n], o) for n in NAMES}
    out = G.storage_from(np.zeros_like(f["utens"]), o)
    G.vadv(*[st[n] for n in NAMES], out, dtr_stage=0.25, prec="df", state48=True)
    G.device_status()
    got = region(out.numpy(), o, (I, J, K)).astype(np.float64)
    ref = region(orc.vadv(*[f[n].astype(np.float64) for n in NAMES], dtr_stage=0.25), o, (I, J, K))
    bad_ref = ~np.all(np.isfinite(ref), axis=0)
    bad_got = ~np.all(np.isfinite(got), axis=0)
    assert bad_ref[0, 2] and np.array_equal(bad_ref, bad_got)
    assert rel_err(got[:, ~bad_ref], ref[:, ~bad_ref]) <= F32_TOL


def test_state48_largest_ensemble_member(G, orc):
    """GTB_STATE48 at the ensemble's largest member shape, 384x384x137 (the longest columns
    and the most live state), within 1e-5 of the FP64 oracle on the FP32-rounded inputs."""
    from paper_2311_08322_b300 import inputs
    I, J, K = 384, 384, 137
    f = {k: v.astype(np.float32) for k, v in inputs.hdiff_vadv(I, J, K, seed=2).items()}
    o = (1, 1, 0)
    st = {n: G.storage_from(f[n], o) for n in NAMES}
    out = G.storage_from(np.zeros_like(f["utens"]), o)
    G.vadv(*[st[n] for n in NAMES], out, prec="df", state48=True)
    G.device_status()
    got = region(out.numpy(), o, (I, J, K))
    ref = region(orc.vadv(*[f[n].astype(np.float64) for n in NAMES]), o, (I, J, K))
    assert rel_err(got, ref) <= F32_TOL
