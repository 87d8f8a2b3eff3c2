"""GPU parity of the spherical-harmonic transforms (paper Sec. 3.2) against the FP64 oracle,
through the C ABI (include/sht.h).  FP64 path: 1e-12 relative (max norm over fields).  The
double-float Legendre precision (SH_DF) is held to the same bounds: its operands carry about 48
significand bits and its sums are compensated dot products, whose error grows like the square
of the FP32 unit (about 1e-13 relative for the sums here), below the FP64 path's 1e-12."""
import numpy as np
import pytest

from oracle import sht as osht

pytestmark = pytest.mark.gpu

A = 6.37122e6
SIZES = [(7, 12, 24), (31, 48, 96), (63, 96, 192), (127, 192, 384)]
# the smallest truncations (one 32-latitude and one 32-degree group, the degree n = T + 1 that
# the vector transforms of the FP64 and double-float plans use next to n = m)
TINY = [(1, 4, 4), (2, 4, 6), (3, 6, 8)]


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


def _rel(x, ref):
    """relative L2 error"""
    return float(np.linalg.norm(x - ref) / np.linalg.norm(ref))


@pytest.mark.parametrize("T,nlat,nlon", SIZES)
def test_grid_matches_oracle(env, T, nlat, nlon):
    torch, rexi = env
    p = rexi.ShPlan(T, nlat, nlon, A)
    mu, w = p.grid()
    omu, ow = osht.gauss_grid(nlat)
    assert np.max(np.abs(mu - omu)) < 1e-14 and np.max(np.abs(w - ow)) < 1e-14
    assert np.max(np.abs(w / ow - 1)) < 1e-11   # relative, the polar weights included
    p.close()


@pytest.mark.parametrize("prec", ["fp64", "df"])
@pytest.mark.parametrize("T,nlat,nlon", TINY + SIZES)
def test_scalar_synthesis_analysis(env, T, nlat, nlon, prec):
    torch, rexi = env
    g = osht.Grid(T, nlat, nlon, A)
    nf = 3
    c = _spec(T, T, nf)
    p = rexi.ShPlan(T, nlat, nlon, A, max_fields=nf, precision=prec)
    cs = torch.from_numpy(c).cuda()
    grid = torch.empty(nf, nlat, nlon, dtype=torch.float64, device="cuda")
    p.synthesis(cs, grid, nf)
    back = torch.empty_like(cs)
    p.analysis(grid, back, nf)
    torch.cuda.synchronize()
    G = grid.cpu().numpy()
    for f in range(nf):
        assert _rel(G[f], g.synth(c[f])) < 1e-12
    # analysis of an arbitrary (not band-limited) grid field against the oracle's analysis
    rng = np.random.default_rng(5)
    f2 = rng.standard_normal((nf, nlat, nlon))
    sp = torch.empty_like(cs)
    p.analysis(torch.from_numpy(f2).cuda(), sp, nf)
    torch.cuda.synchronize()
    S = sp.cpu().numpy()
    for f in range(nf):
        # white noise: large cancellation in every coefficient, so a looser bound
        assert _rel(S[f], g.analys(f2[f])) < 1e-11
    assert _rel(back.cpu().numpy(), c) < 1e-12
    p.close()


@pytest.mark.parametrize("prec", ["fp64", "df"])
@pytest.mark.parametrize("T,nlat,nlon", TINY + SIZES + [(255, 384, 768)])
def test_vector_transforms(env, T, nlat, nlon, prec):
    """Velocity synthesis (the scalar syntheses of the u, v spectra over n = m .. T + 1) and
    divergence / curl (P-sums of A and B, combined over neighbouring degrees) against the
    oracle, which contracts the table of (1 - mu^2) dP/dmu directly."""
    torch, rexi = env
    g = osht.Grid(T, nlat, nlon, A)
    nf = 2
    psi, chi = _spec(T, 1, nf), _spec(T, 2, nf)
    psi[:, 0] = chi[:, 0] = 0
    p = rexi.ShPlan(T, nlat, nlon, A, max_fields=nf, precision=prec)
    U = torch.empty(nf, nlat, nlon, dtype=torch.float64, device="cuda")
    V = torch.empty_like(U)
    p.synthesis_uv(torch.from_numpy(psi).cuda(), torch.from_numpy(chi).cuda(), U, V, nf)
    rng = np.random.default_rng(9)
    Ag, Bg = rng.standard_normal((nf, nlat, nlon)), rng.standard_normal((nf, nlat, nlon))
    dv = torch.empty(nf, osht.nlm(T), dtype=torch.complex128, device="cuda")
    cu = torch.empty_like(dv)
    p.analysis_divcurl(torch.from_numpy(Ag).cuda(), torch.from_numpy(Bg).cuda(), dv, cu, nf)
    torch.cuda.synchronize()
    for f in range(nf):
        Uo, Vo = g.synth_uv(psi[f], chi[f])
        assert _rel(U.cpu().numpy()[f], Uo) < 1e-12
        assert _rel(V.cpu().numpy()[f], Vo) < 1e-12
        do, co = g.analys_divcurl(Ag[f], Bg[f])
        assert _rel(dv.cpu().numpy()[f], do) < 1e-11
        assert _rel(cu.cpu().numpy()[f], co) < 1e-11
    p.close()


@pytest.mark.parametrize("prec", ["fp64", "df"])
def test_T511_sampled(env, prec):
    """Full T511 grid (768 x 1536): synthesis / analysis round trip on the GPU and the
    oracle's synthesis on a few latitudes (its full T511 tables take ~10 s)."""
    torch, rexi = env
    T, nlat, nlon = 511, 768, 1536
    c = _spec(T, 4, 1) * (np.arange(osht.nlm(T)) % 7 + 1.0) ** -1
    p = rexi.ShPlan(T, nlat, nlon, A, precision=prec)
    cs = torch.from_numpy(c).cuda()
    grid = torch.empty(1, nlat, nlon, dtype=torch.float64, device="cuda")
    p.synthesis(cs, grid)
    back = torch.empty_like(cs)
    p.analysis(grid, back)
    torch.cuda.synchronize()
    assert _rel(back.cpu().numpy(), c) < 1e-11
    mu, _ = osht.gauss_grid(nlat)
    rows = [0, 100, 383, 384, 767]
    P = osht.legendre_table(T, mu[rows])
    G = np.zeros((len(rows), T + 1), complex)
    for m in range(T + 1):
        o = osht.moffset(T, m)
        G[:, m] = P[m][:, : T + 1 - m] @ c[0, o: o + T + 1 - m]
    F = np.zeros((len(rows), nlon // 2 + 1), complex)
    F[:, : T + 1] = G
    ref = np.fft.irfft(F, n=nlon, axis=1) * nlon
    assert _rel(grid.cpu().numpy()[0, rows], ref) < 1e-11
    p.close()


def test_errors(env):
    torch, rexi = env
    with pytest.raises(rexi.RexiError):
        rexi.ShPlan(31, 47, 96, A)       # odd nlat
    with pytest.raises(rexi.RexiError):
        rexi.ShPlan(31, 48, 60, A)       # nlon <= 2T
    with pytest.raises(rexi.RexiError):
        rexi.ShPlan(31, 48, 70, A)       # nlon not 2^p 3^q


@pytest.mark.parametrize("scale", [1e-20, 1e20])
def test_double_float_magnitudes(env, scale):
    """SH_DF inside its documented range (the FP32 exponent range): spectra scaled by 1e+-20 give
    the FP64 plan's results to the same relative accuracy (synthesis, analysis of the grids,
    vector transforms); tiny values take the FP64 route of the input split."""
    torch, rexi = env
    T, nlat, nlon, nf = 63, 96, 192, 2
    c = _spec(T, 31, nf) * scale
    psi, chi = _spec(T, 32, 1) * scale, _spec(T, 33, 1) * scale
    psi[:, 0] = chi[:, 0] = 0
    out = {}
    for prec in ("fp64", "df"):
        p = rexi.ShPlan(T, nlat, nlon, A, max_fields=nf, precision=prec)
        cs = torch.from_numpy(c).cuda()
        grid = torch.empty(nf, nlat, nlon, dtype=torch.float64, device="cuda")
        U = torch.empty(1, nlat, nlon, dtype=torch.float64, device="cuda")
        V = torch.empty_like(U)
        p.synthesis(cs, grid, nf)
        p.synthesis_uv(torch.from_numpy(psi).cuda(), torch.from_numpy(chi).cuda(), U, V, 1)
        back = torch.empty_like(cs)
        p.analysis(grid, back, nf)
        dv = torch.empty(1, osht.nlm(T), dtype=torch.complex128, device="cuda")
        cu = torch.empty_like(dv)
        p.analysis_divcurl(U, V, dv, cu, 1)
        p.check()
        out[prec] = [x.cpu().numpy() for x in (grid, U, V, back, dv, cu)]
        p.close()
    for name, a, b in zip(("grid", "U", "V", "spec", "div", "curl"), out["df"], out["fp64"]):
        assert np.all(np.isfinite(a)), name
        assert _rel(a, b) < 1e-12, (name, _rel(a, b))


@pytest.mark.parametrize("prec", ["fp64", "df", "tf32x3"])
def test_plans_of_different_sizes_coexist(env, prec):
    """A small plan created after a large one leaves the large one working: the kernels'
    shared-memory limits are process-wide and only grow (the double-float FFT of 1536 points
    needs 55 KB, the FP32 one 28 KB; a T7 plan's FFT needs under 2 KB).  Round trip of the
    T511 plan after the T7 plan exists, against the band-limited input (exact for the FP64 and
    double-float plans, split TF32 within its 4u = 3.8e-6 per-transform bound, twice)."""
    torch, rexi = env
    big = rexi.ShPlan(511, 768, 1536, A, precision=prec, max_fields=2)
    small = rexi.ShPlan(7, 12, 24, A, precision=prec, max_fields=2)
    for p, (T, nlat, nlon) in ((small, (7, 12, 24)), (big, (511, 768, 1536)), (small, (7, 12, 24))):
        c = _spec(T, 5, 2)
        g = torch.empty(2, nlat, nlon, dtype=torch.float64, device="cuda")
        back = torch.empty(2, osht.nlm(T), dtype=torch.complex128, device="cuda")
        p.synthesis(torch.from_numpy(c).cuda(), g, 2)
        p.analysis(g, back, 2)
        p.check()
        err = _rel(back.cpu().numpy(), c)
        assert err < (1e-12 if prec in ("fp64", "df") else 2 * 3.8e-6), (T, err)
    small.close()
    big.close()
