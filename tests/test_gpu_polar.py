"""Polar truncation of the Legendre sums (include/sht.h, SH_POLAR_THRESHOLD_DEFAULT; the
transforms of paper Sec. 3.2, computed there with SHTns, which skips the same terms).

Pins, through the C ABI:
  * at the default threshold every transform of every precision equals the untruncated plan's
    (polar_threshold < 0) to far below its own rounding;
  * at a large threshold the change obeys the documented bound: every skipped table entry is
    below the threshold, so a synthesised value moves by at most thr x the sum of |c| over the
    terms (times 2 for m > 0, the conjugate half), an analysed coefficient by at most
    thr x sum_j w_j (|F_N| + |F_S|) <= 4 pi thr max|f|;
  * the plan's table counts: needed <= streamed <= total, about three quarters of the T511
    table needed at the default threshold, everything with the truncation off.
The parity tests against the oracle (which never truncates) run with the default threshold."""
import numpy as np
import pytest

from oracle import sht as osht

pytestmark = pytest.mark.gpu

A = 6.37122e6
PRECS = ["fp64", "df", "tf32x3", "tf32", "bf16"]


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1805_06557_gb300 import rexi
    return torch, rexi


def _spec(T, seed, nf=1):
    rng = np.random.default_rng(seed)
    c = rng.standard_normal((nf, osht.nlm(T))) + 1j * rng.standard_normal((nf, osht.nlm(T)))
    c[:, : T + 1] = c[:, : T + 1].real
    return c


def _all_transforms(torch, p, T, nlat, nlon, c, psi, chi, grids):
    """Every transform of the plan on the same inputs: results as numpy arrays."""
    nlm = osht.nlm(T)
    nf = c.shape[0]
    d = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    g = torch.empty(nf, nlat, nlon, dtype=torch.float64, device="cuda")
    U = torch.empty(1, nlat, nlon, dtype=torch.float64, device="cuda")
    V = torch.empty_like(U)
    gm = torch.empty_like(g)
    Um, Vm = torch.empty_like(U), torch.empty_like(U)
    back = torch.empty(nf, nlm, dtype=torch.complex128, device="cuda")
    dv = torch.empty(2, nlm, dtype=torch.complex128, device="cuda")
    cu = torch.empty_like(dv)
    bm = torch.empty_like(back)
    dvm, cum = torch.empty_like(dv), torch.empty_like(dv)
    G = d(grids)
    p.synthesis(d(c), g, nf)
    p.synthesis_uv(d(psi), d(chi), U, V, 1)
    p.synthesis_mixed(d(c), gm, nf, d(psi), d(chi), Um, Vm, 1)
    p.analysis(G[:nf], back, nf)
    p.analysis_divcurl(G[:1], G[1:2], dv[:1], cu[:1], 1)
    p.analysis_mixed(G[:2], G[2:4], dvm, cum, 2, G[:1], bm[:1], 1)
    p.check()
    return {k: v.cpu().numpy() for k, v in dict(g=g, U=U, V=V, gm=gm, Um=Um, Vm=Vm, back=back, dv=dv[:1],
                                                 cu=cu[:1], bm=bm[:1], dvm=dvm, cum=cum).items()}


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("T,nlat,nlon", [(127, 192, 384), (255, 384, 768), (511, 768, 1536)])
def test_default_truncation_equals_full_sums(env, T, nlat, nlon, prec):
    """(At T511 the tensor-core synthesis jobs of the polar latitude tile skip K chunks; at
    T127 and T255 only their analysis jobs do.)"""
    torch, rexi = env
    c = _spec(T, 7, 2) * (np.arange(osht.nlm(T)) % 5 + 1.0) ** -1
    psi, chi = _spec(T, 8), _spec(T, 9)
    psi[:, 0] = chi[:, 0] = 0
    rng = np.random.default_rng(10)
    grids = rng.standard_normal((4, nlat, nlon))
    out = {}
    for thr in (0.0, -1.0):
        p = rexi.ShPlan(T, nlat, nlon, A, precision=prec, max_fields=3, polar_threshold=thr)
        use = p.table_use()
        if thr == 0.0:
            assert use["threshold"] == 1e-19
            assert use["needed_synth"] < use["total"] and use["needed_anal"] < use["total"]
        else:
            assert use["threshold"] == 0.0
            assert use["needed_synth"] == use["needed_anal"] == use["total"]
            assert use["streamed_synth"] == use["streamed_anal"] == use["total"]
        out[thr] = _all_transforms(torch, p, T, nlat, nlon, c, psi, chi, grids)
        p.close()
    # the skipped terms are ~1e-19 of the coefficients, below rounding: FP64 to 1e-14;
    # double-float to 1e-13 (its own accuracy against FP64 is about 1e-14 to 1e-13, and the
    # 1e-12 held against the oracle stays far away); tensor-core precisions below their FP32
    # accumulation's rounding
    tol = {"fp64": 1e-14, "df": 1e-13}.get(prec, 1e-6)
    for k, a in out[0.0].items():
        b = out[-1.0][k]
        assert np.all(np.isfinite(a)), k
        err = np.max(np.abs(a - b)) / np.max(np.abs(b))
        assert err < tol, (prec, k, err)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("T,nlat,nlon", [(127, 192, 384), (255, 384, 768)])
def test_large_threshold_obeys_the_bound(env, T, nlat, nlon, prec):
    """thr = 1e-4: the change of a synthesised grid value stays below
    thr sum_m (1 or 2) sum_n |c_n^m|, of an analysed coefficient below 4 pi thr max|f|; it is
    not zero exactly when the plan streams less than the whole table (the tensor-core
    synthesis tiles of 128 latitudes reach the equator at these sizes and skip nothing; its
    analysis jobs skip K chunks, some all but their last one: TF32 and split TF32 at T127,
    BF16 at T255)."""
    torch, rexi = env
    thr = 1e-4
    c = _spec(T, 11)
    rng = np.random.default_rng(12)
    f = rng.standard_normal((1, nlat, nlon))
    res, uses = {}, {}
    for t in (thr, -1.0):
        p = rexi.ShPlan(T, nlat, nlon, A, precision=prec, polar_threshold=t)
        g = torch.empty(1, nlat, nlon, dtype=torch.float64, device="cuda")
        s = torch.empty(1, osht.nlm(T), dtype=torch.complex128, device="cuda")
        p.synthesis(torch.from_numpy(c).cuda(), g)
        p.analysis(torch.from_numpy(f).cuda(), s)
        p.check()
        res[t] = (g.cpu().numpy(), s.cpu().numpy())
        uses[t] = p.table_use()
        p.close()
    wm = np.ones(osht.nlm(T))
    wm[T + 1:] = 2.0                        # m > 0: the conjugate half doubles the bound
    bound_syn = thr * np.sum(wm * np.abs(c[0]))
    bound_ana = 4 * np.pi * thr * np.max(np.abs(f))
    dg = np.max(np.abs(res[thr][0] - res[-1.0][0]))
    ds = np.max(np.abs(res[thr][1] - res[-1.0][1]))
    # slack for the accumulation rounding of the reduced precisions (identical operands)
    slack_g = 0.0 if prec in ("fp64", "df") else 1e-6 * np.max(np.abs(res[-1.0][0]))
    slack_s = 0.0 if prec in ("fp64", "df") else 1e-6 * np.max(np.abs(res[-1.0][1]))
    u = uses[thr]
    assert dg <= bound_syn + slack_g, (dg, bound_syn)
    assert ds <= bound_ana + slack_s, (ds, bound_ana)
    assert (dg > 0) == (u["streamed_synth"] < u["total"]), (dg, u)
    assert (ds > 0) == (u["streamed_anal"] < u["total"]), (ds, u)
    assert u["needed_synth"] <= u["streamed_synth"] <= u["total"] and u["needed_synth"] < u["total"]
    assert u["needed_anal"] <= u["streamed_anal"] <= u["total"] and u["needed_anal"] < u["total"]
    if prec in ("fp64", "df"):   # whole warps of latitudes / degrees skip at these sizes
        assert u["streamed_synth"] < u["total"] and u["streamed_anal"] < u["total"]


@pytest.mark.parametrize("prec", ["fp64", "df", "tf32x3"])
def test_T511_table_use(env, prec):
    """At T511 on the 768-latitude grid about three quarters of each table is needed at the
    default threshold (element-level count); the kernels stream whole warps (FP64,
    double-float) or whole 128 x chunk tiles (tensor cores), more than needed and less than
    the table."""
    torch, rexi = env
    p = rexi.ShPlan(511, 768, 1536, A, precision=prec)
    u = p.table_use()
    p.close()
    assert u["total"] == osht.nlm(511) * 384
    for d in ("synth", "anal"):
        need, st = u["needed_" + d], u["streamed_" + d]
        assert 0.70 * u["total"] < need < 0.85 * u["total"], (d, need / u["total"])
        assert need <= st < u["total"], (d, need, st)
