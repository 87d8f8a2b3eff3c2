"""Tensor-core (tcgen05) Legendre precisions of the SH transforms against the FP64 oracle.

Per-field bounds (relative L2) are 4u, u the unit of the operands as they reach the tensor
cores, with FP32 accumulation: TF32 (10-bit mantissa, round to nearest) u = 2^-11, bound
1.95e-3; BF16 (7-bit mantissa) u = 2^-8, bound 1.56e-2; split TF32 (operands x_hi + x_lo, three
products a_hi b_lo + a_lo b_hi + a_hi b_hi) u = 2^-20, which covers the dropped a_lo b_lo and
the rounding of both lo parts (3 * 2^-22) plus the FP32 accumulation and the FP32 FFT of those
plans, bound 3.8e-6.  The factor 4 allows the growth of K accumulated rounding errors of
random sign (about sqrt of the number of FP32 additions per accumulator, a few units here).
The measured values are printed by the tests."""
import numpy as np
import pytest

from oracle import sht as osht

pytestmark = pytest.mark.gpu

A = 6.37122e6
BOUND = {"tf32": 4 * 2.0 ** -11, "bf16": 4 * 2.0 ** -8, "tf32x3": 4 * 2.0 ** -20}
SIZES = [(31, 48, 96), (127, 192, 384), (255, 384, 768), (511, 768, 1536)]


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1805_06557_gb300 import rexi
    return torch, rexi


def _spec(T, seed, nf=1, slope=-1.0):
    rng = np.random.default_rng(seed)
    n = np.concatenate([np.arange(m, T + 1) for m in range(T + 1)]).astype(float)
    amp = np.maximum(n, 1.0) ** slope
    c = (rng.standard_normal((nf, osht.nlm(T))) + 1j * rng.standard_normal((nf, osht.nlm(T)))) * amp
    c[:, : T + 1] = c[:, : T + 1].real
    return c


def _rel(x, ref):
    return float(np.linalg.norm(x - ref) / np.linalg.norm(ref))


@pytest.mark.parametrize("prec", ["tf32", "bf16", "tf32x3"])
@pytest.mark.parametrize("T,nlat,nlon", SIZES)
def test_tc_scalar(env, prec, T, nlat, nlon):
    torch, rexi = env
    nf = 2
    c = _spec(T, 3, nf)
    ref64 = rexi.ShPlan(T, nlat, nlon, A, "fp64", max_fields=nf)
    p = rexi.ShPlan(T, nlat, nlon, A, prec, max_fields=nf)
    cs = torch.from_numpy(c).cuda()
    g64 = torch.empty(nf, nlat, nlon, dtype=torch.float64, device="cuda")
    g = torch.empty_like(g64)
    ref64.synthesis(cs, g64, nf)
    p.synthesis(cs, g, nf)
    s64 = torch.empty_like(cs)
    s = torch.empty_like(cs)
    ref64.analysis(g64, s64, nf)
    p.analysis(g64, s, nf)
    p.check()
    G, G64 = g.cpu().numpy(), g64.cpu().numpy()
    S, S64 = s.cpu().numpy(), s64.cpu().numpy()
    if T <= 127:  # the oracle itself for the smaller sizes
        og = osht.Grid(T, nlat, nlon, A)
        assert _rel(G64[0], og.synth(c[0])) < 1e-12
    es = max(_rel(G[f], G64[f]) for f in range(nf))
    ea = max(_rel(S[f], S64[f]) for f in range(nf))
    print("%s T%d synthesis %.2e analysis %.2e" % (prec, T, es, ea))
    assert es < BOUND[prec] and ea < BOUND[prec]
    p.close()
    ref64.close()


@pytest.mark.parametrize("prec", ["tf32", "bf16", "tf32x3"])
@pytest.mark.parametrize("T,nlat,nlon", SIZES[:2])
def test_tc_vector(env, prec, T, nlat, nlon):
    torch, rexi = env
    nf = 2
    og = osht.Grid(T, nlat, nlon, A)
    psi, chi = _spec(T, 5, nf), _spec(T, 6, nf)
    psi[:, 0] = chi[:, 0] = 0
    p = rexi.ShPlan(T, nlat, nlon, A, prec, max_fields=nf)
    U = torch.empty(nf, nlat, nlon, dtype=torch.float64, device="cuda")
    V = torch.empty_like(U)
    p.synthesis_uv(torch.from_numpy(psi).cuda(), torch.from_numpy(chi).cuda(), U, V, nf)
    rng = np.random.default_rng(2)
    Ag = np.stack([og.synth(_spec(T, 11 + f)[0]) for f in range(nf)])
    Bg = np.stack([og.synth(_spec(T, 21 + f)[0]) for f in range(nf)])
    dv = torch.empty(nf, osht.nlm(T), dtype=torch.complex128, device="cuda")
    cu = torch.empty_like(dv)
    p.analysis_divcurl(torch.from_numpy(Ag).cuda(), torch.from_numpy(Bg).cuda(), dv, cu, nf)
    p.check()
    for f in range(nf):
        Uo, Vo = og.synth_uv(psi[f], chi[f])
        do, co = og.analys_divcurl(Ag[f], Bg[f])
        errs = [_rel(U.cpu().numpy()[f], Uo), _rel(V.cpu().numpy()[f], Vo),
                _rel(dv.cpu().numpy()[f], do), _rel(cu.cpu().numpy()[f], co)]
        print("%s T%d uv/divcurl" % (prec, T), ["%.2e" % e for e in errs])
        assert max(errs) < BOUND[prec], errs
    p.close()


@pytest.mark.parametrize("prec", ["tf32", "bf16", "tf32x3"])
@pytest.mark.parametrize("nf", [1, 3, 5, 8])
def test_tc_field_counts_scalar(env, prec, nf):
    """Field counts up to max_fields = 8 on a plan sized for 8: the fused epilogue takes the
    fields two per 8-column group (an odd count leaves the last group half used), and a call
    writes only its own fields (the rest of the output keeps a sentinel)."""
    torch, rexi = env
    T, nlat, nlon = 63, 96, 192
    og = osht.Grid(T, nlat, nlon, A)
    p = rexi.ShPlan(T, nlat, nlon, A, prec, max_fields=8)
    c = _spec(T, 30 + nf, nf)
    g = torch.full((8, nlat, nlon), 7.0, dtype=torch.float64, device="cuda")
    p.synthesis(torch.from_numpy(c).cuda(), g, nf)
    grids = np.stack([og.synth(c[f]) for f in range(nf)])
    s = torch.full((8, osht.nlm(T)), 7.0 + 0j, dtype=torch.complex128, device="cuda")
    p.analysis(torch.from_numpy(grids).cuda(), s, nf)
    p.check()
    G, S = g.cpu().numpy(), s.cpu().numpy()
    for f in range(nf):
        es, ea = _rel(G[f], grids[f]), _rel(S[f], og.analys(grids[f]))
        assert es < BOUND[prec] and ea < BOUND[prec], (f, es, ea)
    assert np.all(G[nf:] == 7.0) and np.all(S[nf:] == 7.0)
    p.close()


@pytest.mark.parametrize("prec", ["tf32", "bf16", "tf32x3"])
@pytest.mark.parametrize("nf", [1, 3, 4, 8])
def test_tc_field_counts_vector(env, prec, nf):
    """Vector field counts: one 8-column group per field, the (P, H) job pairs of every
    (m, tile) combined in the epilogue; nf = 8 fills 64 columns (two accumulator buffers in
    TMEM) (T = 63, 96 x 192 grid)."""
    torch, rexi = env
    T, nlat, nlon = 63, 96, 192
    og = osht.Grid(T, nlat, nlon, A)
    p = rexi.ShPlan(T, nlat, nlon, A, prec, max_fields=max(nf, 4))
    psi, chi = _spec(T, 40 + nf, nf), _spec(T, 50 + nf, nf)
    psi[:, 0] = chi[:, 0] = 0
    U = torch.empty(nf, nlat, nlon, dtype=torch.float64, device="cuda")
    V = torch.empty_like(U)
    p.synthesis_uv(torch.from_numpy(psi).cuda(), torch.from_numpy(chi).cuda(), U, V, nf)
    Ag = np.stack([og.synth(_spec(T, 60 + f)[0]) for f in range(nf)])
    Bg = np.stack([og.synth(_spec(T, 70 + f)[0]) for f in range(nf)])
    dv = torch.empty(nf, osht.nlm(T), dtype=torch.complex128, device="cuda")
    cu = torch.empty_like(dv)
    p.analysis_divcurl(torch.from_numpy(Ag).cuda(), torch.from_numpy(Bg).cuda(), dv, cu, nf)
    p.check()
    for f in range(nf):
        Uo, Vo = og.synth_uv(psi[f], chi[f])
        do, co = og.analys_divcurl(Ag[f], Bg[f])
        errs = [_rel(U.cpu().numpy()[f], Uo), _rel(V.cpu().numpy()[f], Vo),
                _rel(dv.cpu().numpy()[f], do), _rel(cu.cpu().numpy()[f], co)]
        assert max(errs) < BOUND[prec], (f, errs)
    p.close()


@pytest.mark.parametrize("prec", ["tf32", "tf32x3"])
def test_tc_gemm_timeout_path_reports_etimeout(env, prec):
    """The bounded-wait error path of the tensor-core GEMM, run for real: a plan whose epilogue
    gives up after one non-blocking poll of its accumulator barrier (the MMAs cannot have
    completed by then: the B operand and the first A chunk are still in flight) records the
    error, the kernel still ends (copies and MMAs drain with their full bounds; with one job
    per CTA the MMA warp never waits for the epilogue), sh_plan_check reports REXI_ETIMEOUT,
    and a following plan of the same precision transforms correctly."""
    torch, rexi = env
    T, nlat, nlon, nf = 15, 24, 48, 1
    c = _spec(T, 7, nf)
    cs = torch.from_numpy(c).cuda()
    g = torch.empty(nf, nlat, nlon, dtype=torch.float64, device="cuda")
    bad = rexi.ShPlan(T, nlat, nlon, A, prec, max_fields=nf, epilogue_wait_polls=1)
    bad.synthesis(cs, g, nf)
    with pytest.raises(rexi.RexiError) as e:
        bad.check()
    assert e.value.code == rexi.REXI_ETIMEOUT
    bad.close()
    good = rexi.ShPlan(T, nlat, nlon, A, prec, max_fields=nf)
    good.synthesis(cs, g, nf)
    good.check()
    og = osht.Grid(T, nlat, nlon, A)
    assert _rel(g.cpu().numpy()[0], og.synth(c[0])) < BOUND[prec]
    good.close()


MIXED = [(31, 48, 96, 4, 2, 1), (31, 48, 96, 4, 1, 2), (31, 48, 96, 4, 3, 2), (31, 48, 96, 4, 1, 3),
         (127, 192, 384, 3, 1, 1), (511, 768, 1536, 3, 2, 1), (511, 768, 1536, 3, 1, 2)]


@pytest.mark.parametrize("prec", ["fp64", "tf32", "bf16", "tf32x3", "df"])
@pytest.mark.parametrize("T,nlat,nlon,mf,nfs,nfv", MIXED)
def test_mixed_transforms_equal_separate_calls(env, prec, T, nlat, nlon, mf, nfs, nfv):
    """sh_synthesis_mixed / sh_analysis_mixed (nfs scalar fields beside nfv vector pairs, one
    read of each table) give the results of the separate scalar and vector calls bit for bit:
    every accumulator column depends on its own B column only, and the epilogue combines the
    same sums in the same order.  Includes the nonlinear term's combinations (2 scalar + 1
    vector synthesis, 2 vector + 1 scalar analysis) at T511."""
    torch, rexi = env
    p = rexi.ShPlan(T, nlat, nlon, A, prec, max_fields=mf)
    cs = torch.from_numpy(_spec(T, 21, nfs)).cuda()
    psi = torch.from_numpy(_spec(T, 22, nfv, -2.0)).cuda()
    chi = torch.from_numpy(_spec(T, 23, nfv, -2.0)).cuda()
    grid = lambda n: torch.empty(n, nlat, nlon, dtype=torch.float64, device="cuda")
    g1, U1, V1 = grid(nfs), grid(nfv), grid(nfv)
    g2, U2, V2 = grid(nfs), grid(nfv), grid(nfv)
    p.synthesis(cs, g1, nfs)
    p.synthesis_uv(psi, chi, U1, V1, nfv)
    p.synthesis_mixed(cs, g2, nfs, psi, chi, U2, V2, nfv)
    s1, d1, c1 = torch.empty_like(cs), torch.empty_like(psi), torch.empty_like(psi)
    s2, d2, c2 = torch.empty_like(cs), torch.empty_like(psi), torch.empty_like(psi)
    p.analysis(g1, s1, nfs)
    p.analysis_divcurl(U1, V1, d1, c1, nfv)
    p.analysis_mixed(U1, V1, d2, c2, nfv, g1, s2, nfs)
    p.check()
    for name, a, b in (("grid", g1, g2), ("U", U1, U2), ("V", V1, V2), ("spec", s1, s2), ("div", d1, d2),
                       ("curl", c1, c2)):
        assert torch.isfinite(torch.view_as_real(a) if a.is_complex() else a).all(), name
        assert torch.equal(a, b), (name, float((a - b).abs().max()), float(a.abs().max()))
    p.close()


def test_mixed_transform_limits(env):
    torch, rexi = env
    p = rexi.ShPlan(31, 48, 96, A, "tf32", max_fields=2)
    z = torch.zeros(4, osht.nlm(31), dtype=torch.complex128, device="cuda")
    g = torch.zeros(4, 48, 96, dtype=torch.float64, device="cuda")
    with pytest.raises(rexi.RexiError):
        p.synthesis_mixed(z, g, 1, z, z, g, g, 2)     # 1 + 2 x 2 > 2 max_fields
    with pytest.raises(rexi.RexiError):
        p.analysis_mixed(g, g, z, z, 0, g, z, 1)      # no vector pair
    p.close()
