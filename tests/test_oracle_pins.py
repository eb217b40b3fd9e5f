"""Pins of the FP64 oracle against facts that do not come from the oracle itself:
finite differences of its own energies, closed forms, an independent Philox
implementation, torch.autograd, invariants and brute force on tiny inputs.
CPU only (no GPU marker)."""
import math
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2408_14070_gb300 import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))


# --------------------------------------------------------------------------- Philox
def test_philox_matches_triton_interpreter(orc, tmp_path):
    pytest.importorskip("triton")
    rng = np.random.default_rng(7)
    ctr = rng.integers(0, 2 ** 32, size=(200, 4), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    ctr[1] = 0xFFFFFFFF
    ctr[2] = [1, 0, 0, 0]
    seed = 0x0123456789ABCDEF
    np.save(tmp_path / "c.npy", ctr)
    subprocess.run([sys.executable, os.path.join(HERE, "philox_triton_ref.py"), str(tmp_path / "c.npy"),
                    str(seed), str(tmp_path / "o.npy")], check=True, timeout=600)
    ref = np.load(tmp_path / "o.npy")
    got = orc.philox(ctr, seed)
    assert np.array_equal(got, ref)
    # the key matters in both halves
    assert not np.array_equal(orc.philox(ctr, seed ^ 1), got)
    assert not np.array_equal(orc.philox(ctr, seed ^ (1 << 40)), got)


def test_normals_are_standard_gaussian(orc):
    from scipy import stats
    n = 100_000
    idx = np.arange(n, dtype=np.uint32)
    bwss = np.stack([idx % 977, idx // 977, np.full(n, 12345, np.uint32), np.zeros(n, np.uint32)], 1)
    z = orc.normals(bwss, seed=99)
    for k in range(3):
        assert abs(z[:, k].mean()) < 5 / math.sqrt(n)
        assert abs(z[:, k].var() - 1) < 5 * math.sqrt(2 / n)
        assert stats.kstest(z[:, k], "norm").pvalue > 1e-4
    c = np.corrcoef(z.T)
    assert np.abs(c - np.eye(3)).max() < 5 / math.sqrt(n)
    # distinct streams and steps give different draws
    b2 = bwss.copy(); b2[:, 3] = 1
    assert np.abs(orc.normals(b2[:10], 99) - z[:10]).min() > 0


def fma32(a, b, c):
    """Correctly rounded float32 fused multiply-add, from exact rational
    arithmetic (round to nearest, ties to even)."""
    from fractions import Fraction
    a, b, c = np.float32(a), np.float32(b), np.float32(c)
    q = Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c))
    f = np.float32(float(q))
    cands = [np.nextafter(f, np.float32(-np.inf)), f, np.nextafter(f, np.float32(np.inf))]

    def key(x):
        odd = int(np.frombuffer(np.float32(x).tobytes(), np.uint32)[0]) & 1
        return (abs(Fraction(float(x)) - q), odd)
    return np.float32(min(cands, key=key))


def r2_fma(d):
    """r^2 as the kernel forms it: fma(dz, dz, fma(dy, dy, dx dx)), FP32."""
    d = d.astype(np.float32)
    return fma32(d[2], d[2], fma32(d[1], d[1], np.float32(d[0] * d[0])))


def test_fma32_emulation_against_float64_where_exact():
    rng = np.random.default_rng(3)
    for _ in range(200):
        a, b, c = (np.float32(v) for v in rng.normal(size=3))
        # a*b is exact in float64 (24 + 24 bits), so float64 a*b + c rounded to
        # float32 differs from the true fma only on double-rounding ties
        ref = np.float32(float(a) * float(b) + float(c))
        got = fma32(a, b, c)
        assert abs(float(got) - float(ref)) <= float(np.spacing(np.float32(abs(ref)) if ref != 0 else np.float32(1e-38)))
    assert fma32(np.float32(1 + 2 ** -23), np.float32(1 - 2 ** -23), np.float32(-1)) == np.float32(-2.0 ** -46)


# --------------------------------------------------------------------------- geometry
def test_dihedral_sign_convention_and_ties(orc):
    # looking down the p1->p2 axis, p0 projects on +x, p3 on +y: IUPAC +90 deg
    p = np.array([[1, 0, 0], [0, 0, 0], [0, 0, 1], [0, 1, 1]], float)
    assert orc.dihedral(p)[0] == pytest.approx(math.pi / 2, abs=1e-14)
    q = p.copy(); q[3] = [0, -1, 1]
    assert orc.dihedral(q)[0] == pytest.approx(-math.pi / 2, abs=1e-14)
    cis = np.array([[1, 0, 0], [0, 0, 0], [0, 0, 1], [1, 0, 1]], float)
    assert orc.dihedral(cis)[0] == pytest.approx(0.0, abs=1e-14)
    trans = np.array([[1, 0, 0], [0, 0, 0], [0, 0, 1], [-1, 0, 1]], float)
    assert orc.dihedral(trans)[0] == -math.pi      # half-open [-pi, pi)
    # rigid-motion invariance
    rng = np.random.default_rng(1)
    pts = rng.normal(size=(4, 3))
    qm, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(qm) < 0:
        qm[:, 0] *= -1
    assert orc.dihedral(pts @ qm.T + 3.0)[0] == pytest.approx(orc.dihedral(pts)[0], abs=1e-12)
    # a mirror image flips the sign
    assert orc.dihedral(pts * np.array([1, 1, -1]))[0] == pytest.approx(-orc.dihedral(pts)[0], abs=1e-12)


def test_wrap_pi(orc):
    assert orc.wrap_pi(math.pi) == -math.pi
    assert orc.wrap_pi(-math.pi) == -math.pi
    assert orc.wrap_pi(3 * math.pi) == pytest.approx(-math.pi)
    for d in np.linspace(-20, 20, 101):
        w = orc.wrap_pi(d)
        assert -math.pi <= w < math.pi
        assert abs(math.remainder(d - w, 2 * math.pi)) < 1e-12


def _fd_forces(fun, x, h=1e-6):
    g = np.zeros_like(x)
    for i in range(x.shape[0]):
        for k in range(3):
            xp = x.copy(); xp[i, k] += h
            xm = x.copy(); xm[i, k] -= h
            g[i, k] = -(fun(xp) - fun(xm)) / (2 * h)
    return g


@pytest.mark.parametrize("n,seed", [(22, 1), (22, 2), (60, 3)])
def test_force_field_equals_minus_gradient(orc, n, seed):
    sp = I.make_system(n, 4, seed)
    x = I.make_chains(1, sp, seed)[0].astype(np.float64)
    U, f, terms = orc.ff(sp, x)
    assert U == pytest.approx(terms.sum())
    assert terms[3] != 0.0 and terms[2] != 0.0
    fd = _fd_forces(lambda y: orc.ff(sp, y, forces=False)[0], x)
    assert np.abs(fd - f).max() <= 1e-7 * np.abs(f).max()
    # translation invariance: forces sum to zero
    assert np.abs(f.sum(0)).max() < 1e-9 * np.abs(f).max()


def test_force_field_terms_fd_at_stretched_geometry(orc):
    # stretch bonds and bend angles away from their minima so every term has force
    sp = I.make_system(12, 2, 5)
    x = I.make_chains(1, sp, 5)[0].astype(np.float64) * 1.07
    x += np.random.default_rng(0).normal(scale=0.03, size=x.shape)
    U, f, terms = orc.ff(sp, x)
    assert min(abs(terms[0]), abs(terms[1])) > 1e-3
    fd = _fd_forces(lambda y: orc.ff(sp, y, forces=False)[0], x)
    assert np.abs(fd - f).max() <= 1e-7 * np.abs(f).max()


def test_cv_jacobian_matches_finite_differences(orc):
    sp = I.make_system(40, 9, 4)
    x = I.make_chains(1, sp, 4)[0].astype(np.float64)
    s, J = orc.cvs(sp, x)
    h = 1e-6
    for j in range(sp.n_cv):
        for a in range(4):
            at = sp.cv_atoms[j, a]
            for k in range(3):
                xp = x.copy(); xp[at, k] += h
                xm = x.copy(); xm[at, k] -= h
                d = orc.wrap_pi(orc.cvs(sp, xp)[0][j] - orc.cvs(sp, xm)[0][j]) / (2 * h)
                assert abs(d - J[j, a, k]) < 1e-7 * max(1.0, abs(J[j]).max())


def test_lj_pair_set_bruteforce_fp32_strict_cutoff(orc):
    # eight beads on a line with one pair placed exactly at the cutoff (in FP32)
    rc = 2.5
    x = np.zeros((8, 3), np.float32)
    x[:, 0] = np.array([0.0, 1.0, 2.0, 2.5, 3.4, 4.9, 6.0, 7.3], np.float32)
    x[:, 1] = np.array([0, 0.3, 0, 0.0, 0.1, 0, 0.4, 0], np.float32)
    # hand enumeration of the candidate pairs |i - j| >= 3 with the FP32 r^2
    rc2 = np.float32(rc * rc)
    want = []
    for i in range(8):
        for j in range(i + 3, 8):
            if r2_fma(x[j] - x[i]) < rc2:
                want.append((i, j))
    got = [tuple(p) for p in orc.lj_pairs(x, rc)]
    assert got == want
    assert (0, 3) not in got          # r = 2.5 exactly: excluded by the strict test
    assert (1, 4) in got and (2, 5) not in got


def test_lj_pair_decision_follows_the_fused_form(orc):
    """Search pairs whose r^2 lands within a few ulp of rc^2, where the fused
    and unfused FP32 forms can disagree; the oracle must follow the fused one."""
    rng = np.random.default_rng(11)
    rc = 2.5
    rc2 = np.float32(rc * rc)
    found = 0
    for _ in range(20000):
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        d = (u * rc * (1 + rng.uniform(-3e-7, 3e-7))).astype(np.float32)
        fused = r2_fma(d)
        plain = np.float32(np.float32(np.float32(d[0] * d[0]) + np.float32(d[1] * d[1])) + np.float32(d[2] * d[2]))
        if (fused < rc2) != (plain < rc2):
            x = np.zeros((4, 3), np.float32)
            x[3] = d
            assert len(orc.lj_pairs(x, rc)) == int(fused < rc2)
            found += 1
            if found >= 5:
                break
    assert found >= 1


def test_lj_pairs_random_chain_bruteforce(orc):
    sp = I.make_system(30, 2, 8)
    x = I.make_chains(1, sp, 8)[0]
    rc2 = np.float32(sp.lj_rc * sp.lj_rc)
    want = []
    for i in range(30):
        for j in range(i + 3, 30):
            if r2_fma((x[j] - x[i]).astype(np.float32)) < rc2:
                want.append((i, j))
    assert [tuple(p) for p in orc.lj_pairs(x, sp.lj_rc)] == want


# --------------------------------------------------------------------------- ensemble
def _torch_member(ens, m, u):
    torch = pytest.importorskip("torch")
    D, L, H = ens.n_in, ens.n_layers, ens.width
    w = torch.tensor(ens.weights[m].astype(np.float64))
    uu = torch.tensor(u, dtype=torch.float64, requires_grad=True)
    p, h = 0, uu
    for l in range(L):
        fin = D if l == 0 else H
        W = w[p:p + H * fin].reshape(H, fin); p += H * fin
        b = w[p:p + H]; p += H
        t = torch.tanh(W @ h + b)
        h = t + h if (ens.resnet and l > 0) else t
    A = w[p:p + H] @ h + w[p + H]
    (g,) = torch.autograd.grad(A, uu)
    return float(A.detach()), g.numpy()


@pytest.mark.parametrize("resnet", [False, True])
def test_mlp_value_and_input_gradient_vs_autograd(orc, resnet):
    ens = I.make_ensemble(3, 10, 3, 32, 2, resnet=resnet)
    rng = np.random.default_rng(3)
    for m in range(3):
        u = rng.uniform(-1, 1, size=10)
        A, g = orc.mlp(ens, m, u)
        At, gt = _torch_member(ens, m, u)
        assert A == pytest.approx(At, rel=1e-12, abs=1e-12)
        assert np.allclose(g, gt, rtol=1e-11, atol=1e-13)


def test_ensemble_gradient_on_cvs_vs_autograd(orc):
    torch = pytest.importorskip("torch")
    ens = I.make_ensemble(4, 8, 2, 16, 4)
    s = np.random.default_rng(4).uniform(-math.pi, math.pi, 4)
    r = orc.ensemble(ens, s)
    for m in range(4):
        st = torch.tensor(s, requires_grad=True)
        u = torch.stack([torch.cos(st), torch.sin(st)], 1).reshape(-1)
        D, L, H = 8, 2, 16
        w = torch.tensor(ens.weights[m].astype(np.float64))
        p, h = 0, u
        for l in range(L):
            fin = D if l == 0 else H
            W = w[p:p + H * fin].reshape(H, fin); p += H * fin
            b = w[p:p + H]; p += H
            h = torch.tanh(W @ h + b)
        A = w[p:p + H] @ h + w[p + H]
        (g,) = torch.autograd.grad(A, st)
        assert np.allclose(r["gradA"][m], g.numpy(), rtol=1e-11, atol=1e-13)


def test_model_deviation_special_cases(orc):
    base = I.make_ensemble(1, 6, 2, 16, 5)
    s = np.array([0.3, -1.2, 2.5])
    # identical members: eps = 0, so sigma = 1 and F_s = mean force
    same = I.EnsembleParams(4, 6, 2, 16, False, np.repeat(base.weights, 4, 0), 0.1, 0.2)
    r = orc.ensemble(same, s)
    assert r["eps"] == pytest.approx(0.0, abs=1e-14) and r["sigma"] == 1.0
    assert np.allclose(r["Fs"], r["gradA"][0])
    one = I.EnsembleParams(1, 6, 2, 16, False, base.weights, 0.1, 0.2)
    assert orc.ensemble(one, s)["eps"] == 0.0
    # two members whose output layers differ by a factor alpha: g2 = alpha g1,
    # so Fbar = (1 + alpha)/2 g1 and eps = |1 - alpha|/2 |g1|
    alpha = 0.4
    w2 = np.repeat(base.weights, 2, 0).copy()
    P = w2.shape[1]
    w2[1, P - 17:P - 1] *= alpha
    two = I.EnsembleParams(2, 6, 2, 16, False, w2, 1e9, 2e9)
    r2 = orc.ensemble(two, s)
    g1 = r2["gradA"][0]
    assert np.allclose(r2["gradA"][1], alpha * g1, rtol=1e-6, atol=1e-6)
    assert r2["eps"] == pytest.approx(abs(1 - alpha) / 2 * np.linalg.norm(g1), rel=1e-6)
    assert np.allclose(r2["Fs"], (1 + alpha) / 2 * g1, rtol=1e-6, atol=1e-7)


def test_switch_properties(orc):
    e0, e1 = 2.0, 3.0
    assert orc.switch(0.0, e0, e1) == 1.0
    assert orc.switch(1.999999, e0, e1) == 1.0
    assert orc.switch(e0, e0, e1) == pytest.approx(1.0)
    assert orc.switch(e1, e0, e1) == 0.0
    assert orc.switch(7.0, e0, e1) == 0.0
    assert orc.switch(2.5, e0, e1) == pytest.approx(0.5)
    xs = np.linspace(e0, e1, 41)
    vals = np.array([orc.switch(v, e0, e1) for v in xs])
    assert np.all(np.diff(vals) <= 0)
    # symmetric about the midpoint and flat (zero slope) at both ends
    for t in np.linspace(0, 0.5, 11):
        assert orc.switch(e0 + t, e0, e1) + orc.switch(e1 - t, e0, e1) == pytest.approx(1.0, abs=1e-12)
    h = 1e-4
    assert abs(orc.switch(e0 + h, e0, e1) - 1.0) < 1e-6
    assert abs(orc.switch(e1 - h, e0, e1)) < 1e-6


def test_bias_force_is_minus_gradient_of_bias_potential(orc):
    """With sigma = 1 the bias potential is -Abar(s(x)); its negative gradient
    must equal the chain-ruled bias force on the beads."""
    sp = I.make_system(30, 5, 6)
    x = I.make_chains(1, sp, 6)[0].astype(np.float64)
    ens = I.make_ensemble(4, 10, 2, 32, 6, trust_lo=1e9, trust_hi=2e9)
    rb = orc.total(sp, x, ens=ens, mode=1)
    r0 = orc.total(sp, x, mode=0)
    fb = rb["f"] - r0["f"]
    assert np.abs(fb).max() > 1e-3
    fd = _fd_forces(lambda y: -orc.total(sp, y, ens=ens, mode=1)["Abar"], x)
    assert np.abs(fd - fb).max() <= 1e-6 * np.abs(fb).max()


def test_switched_bias_scales_with_sigma(orc):
    sp = I.make_system(30, 5, 6)
    x = I.make_chains(1, sp, 6)[0].astype(np.float64)
    ens = I.make_ensemble(4, 10, 2, 32, 6, trust_lo=1e9, trust_hi=2e9)
    full = orc.total(sp, x, ens=ens)["f"] - orc.total(sp, x)["f"]
    eps = orc.ensemble(ens, orc.cvs(sp, x)[0])["eps"]
    for e0, e1, sig in [(eps - 1.0, eps + 1.0, 0.5), (eps + 1e-3, eps + 1, 1.0), (eps - 2, eps - 1, 0.0)]:
        ens.trust_lo, ens.trust_hi = e0, e1
        part = orc.total(sp, x, ens=ens)["f"] - orc.total(sp, x)["f"]
        assert np.allclose(part, sig * full, atol=1e-12)


def test_restraint_force_is_minus_gradient(orc):
    sp = I.make_system(30, 5, 9)
    x = I.make_chains(1, sp, 9)[0].astype(np.float64)
    s0 = I.make_label_targets(1, 5, 9)[0]
    kap = np.array([50.0, 80.0, 120.0, 300.0, 500.0])
    fr = orc.total(sp, x, mode=2, s0=s0, kappa=kap)["f"] - orc.total(sp, x)["f"]
    fd = _fd_forces(lambda y: orc.total(sp, y, mode=2, s0=s0, kappa=kap)["U_restraint"], x)
    assert np.abs(fd - fr).max() <= 1e-6 * np.abs(fr).max()


# --------------------------------------------------------------------------- dynamics
def test_nve_energy_error_bounded_and_second_order(orc):
    """gamma = 0 (velocity Verlet): the total energy error stays small and falls
    roughly as dt^2 (a first-order slip, e.g. a missing half kick, fails)."""
    med = []
    x0 = None
    for dt, n in [(0.005, 10000), (0.00125, 40000)]:
        sp = I.make_system(22, 2, 1, gamma=0.0, dt=dt, output_freq=int(round(0.05 / dt)))
        if x0 is None:
            x0 = I.make_chains(8, sp, 1)
        ens = I.make_ensemble(4, 4, 3, 64, 1, trust_lo=1e9, trust_hi=2e9)
        r = orc.explore(sp, x0, n, ens=ens, energy=True)
        E = r["energy"].sum(-1)
        dev = np.abs(E - E[:, :1]).max(axis=1) / (3 * sp.n_beads * sp.kT)
        if dt == 0.005:
            assert dev.max() < 2e-3
        med.append(np.median(dev))
    assert med[0] / med[1] > 6.0


def test_baoab_exact_harmonic_configurational_variance(orc):
    # BAOAB samples the exact Boltzmann variance kT/a of a harmonic well at any stable dt
    for dt in (0.3, 0.9):
        r = orc.harmonic1d(a=1.0, c=0.0, kappa=0.0, s0=0.0, n_steps=2_000_000, n_equil=1000, dt=dt, seed=11)
        assert r["mean2"] == pytest.approx(1.0, abs=0.015)
    # a stiffer well at a smaller step, kT = 2
    r = orc.harmonic1d(a=4.0, c=0.5, kappa=0.0, s0=0.0, n_steps=1_000_000, n_equil=1000, dt=0.2, kT=2.0, seed=12)
    assert r["mean"] == pytest.approx(0.5, abs=0.02)
    assert r["mean2"] - r["mean"] ** 2 == pytest.approx(0.5, rel=0.03)


def test_restrained_mean_force_closed_form(orc):
    """1-D harmonic free energy A(s) = a/2 (s - c)^2 under a restraint kappa:
    MF = kappa a (s0 - c)/(a + kappa) (exact for BAOAB's configurational sampling)."""
    z = []
    for seed, (a, c, kap, s0) in enumerate([(2.0, 0.3, 50.0, 1.0), (5.0, -0.4, 500.0, 0.2),
                                            (1.0, 0.0, 10.0, -1.5)]):
        r = orc.harmonic1d(a=a, c=c, kappa=kap, s0=s0, n_steps=1_000_000, n_equil=2000,
                           dt=min(0.02, 0.5 / math.sqrt(a + kap)), seed=20 + seed)
        want = kap * a * (s0 - c) / (a + kap)
        z.append((r["mf"] - want) / r["se"])
    z = np.array(z)
    assert np.all(np.abs(z) < 3.5) and np.mean(z ** 2) < 6.0


def test_label_statistics_block_standard_error(orc):
    rng = np.random.default_rng(2)
    K, B = 100_003, 20
    # iid samples: SE = std/sqrt(K)
    d = rng.normal(0.1, 0.5, size=(K, 2))
    r = orc.label_stats(d, np.array([3.0, 1.0]), B)
    assert np.allclose(r["mf"], -np.array([3.0, 1.0]) * d.mean(0), rtol=1e-12)
    assert np.allclose(r["std"], np.array([3.0, 1.0]) * d.std(0), rtol=1e-9)
    se_true = np.array([3.0, 1.0]) * 0.5 / math.sqrt(K)
    assert np.all(np.abs(r["se"] / se_true - 1) < 0.6)
    # AR(1) samples: the block SE tracks the inflated SE sqrt((1 + rho)/(1 - rho)) sigma/sqrt(K)
    rho = 0.9
    e = rng.normal(size=K)
    y = np.empty(K)
    y[0] = e[0]
    for k in range(1, K):
        y[k] = rho * y[k - 1] + math.sqrt(1 - rho * rho) * e[k]
    r = orc.label_stats(y[:, None], np.array([1.0]), B)
    se_true = math.sqrt((1 + rho) / (1 - rho)) / math.sqrt(K)
    assert 0.5 < r["se"][0] / se_true < 1.6


def test_langevin_chain_equipartition(orc):
    sp = I.make_system(22, 2, 3, output_freq=10)
    x0 = I.make_chains(8, sp, 3)
    r = orc.explore(sp, x0, 4000, energy=True)
    ke = r["energy"][:, 100:, 2]                 # discard the first 1000 steps
    T = ke.mean() * 2 / (3 * sp.n_beads)
    assert T == pytest.approx(sp.kT, rel=0.05)


def test_maxwell_boltzmann_start_and_resume_bitwise(orc):
    sp = I.make_system(22, 2, 4, output_freq=5)
    x0 = I.make_chains(3, sp, 4)
    full = orc.explore(sp, x0, 40)
    a = orc.explore(sp, x0, 20)
    b = orc.explore(sp, a["x"].astype(np.float32), 20, v0=a["v"].astype(np.float32), step0=20)
    # resuming from an FP32 snapshot changes the state by rounding only
    assert np.abs(b["x"] - full["x"]).max() < 1e-4
    assert np.array_equal(full["cv"][:, :4], a["cv"])


# --------------------------------------------------------------------------- non-unit physics
# (m, kT) pairs: kT = 2.49 is R T at 300 K in kJ/mol (the configuration loader's
# default); the second pair puts kT/m far from 1, so that kT/m used for
# sqrt(kT/m), or m and kT swapped, also changes every moment below.
PHYS = [(2.5, 2.49), (3.0, 0.6), (0.4, 2.49)]


@pytest.mark.parametrize("m,kT", PHYS)
def test_maxwell_boltzmann_start_has_variance_kT_over_m(orc, m, kT):
    """Maxwell-Boltzmann start (reading: Philox stream 1 at step0) over 10^5
    beads: each velocity component has mean 0 and variance kT/m within 5 sigma,
    Gaussian tails (fourth moment 3 (kT/m)^2), and no correlation between
    neighbouring beads, components or walkers."""
    sp = I.make_system(200, 2, 31, mass=m, kT=kT)
    x0 = I.make_chains(500, sp, 31, min_dist=1.0)
    v = orc.explore(sp, x0, 0)["v"]                  # zero steps: the drawn start
    var0 = kT / m
    n = v.shape[0] * v.shape[1]
    for k in range(3):
        c = v[..., k].ravel()
        assert abs(c.mean()) < 5 * math.sqrt(var0 / n)
        assert abs(c.var() - var0) < 5 * var0 * math.sqrt(2.0 / n)
        # Var(c^4) = (105 - 9) var0^4 for a Gaussian
        assert abs(np.mean(c ** 4) - 3 * var0 ** 2) < 5 * math.sqrt(96.0 / n) * var0 ** 2
    for a, b in [(v[:, :-1, :], v[:, 1:, :]), (v[..., 0], v[..., 1]), (v[:-1], v[1:])]:
        a, b = a.ravel(), b.ravel()
        assert abs(np.mean(a * b)) / var0 < 5 / math.sqrt(a.size)
    # the start is not the O-step noise of step 0 (stream 0)
    xi0 = orc.normals(np.array([[i, 0, 0, 0] for i in range(200)]), sp.seed)
    assert not np.allclose(v[0], math.sqrt(var0) * xi0)


@pytest.mark.parametrize("m,kT", PHYS)
def test_baoab_harmonic_variance_at_non_unit_mass(orc, m, kT):
    """BAOAB's configurational variance of a harmonic well is kT/a at any
    stable dt, whatever the mass: a dropped 1/m in a kick, or kT/m in the
    noise amplitude instead of its square root, moves it by a factor m or
    kT/m."""
    a = 3.0
    dt = 0.5 * math.sqrt(m / a)            # omega dt = 0.5
    r = orc.harmonic1d(a=a, c=0.2, kappa=0.0, s0=0.0, n_steps=1_000_000, n_equil=1000, dt=dt, m=m, kT=kT,
                       gamma=0.5, seed=41)
    assert r["mean"] == pytest.approx(0.2, abs=0.03 * math.sqrt(kT / a))
    assert r["mean2"] - r["mean"] ** 2 == pytest.approx(kT / a, rel=0.03)


@pytest.mark.parametrize("m,kT", PHYS)
def test_restrained_mean_force_closed_form_at_non_unit_mass(orc, m, kT):
    """The restrained 1-D mean force kappa a (s0 - c)/(a + kappa) holds for any
    mass and temperature (the configurational distribution does not depend on
    m); its spread, std = kappa sqrt(kT/(a + kappa)), does depend on kT."""
    a, c, kap, s0 = 2.0, 0.3, 50.0, 1.0
    r = orc.harmonic1d(a=a, c=c, kappa=kap, s0=s0, n_steps=1_000_000, n_equil=2000, m=m, kT=kT,
                       dt=0.4 * math.sqrt(m / (a + kap)), gamma=0.5, seed=43)
    want = kap * a * (s0 - c) / (a + kap)
    assert abs(r["mf"] - want) < 3.5 * r["se"]
    assert r["std"] == pytest.approx(kap * math.sqrt(kT / (a + kap)), rel=0.02)


@pytest.mark.parametrize("m,kT", PHYS)
def test_langevin_chain_equipartition_at_non_unit_physics(orc, m, kT):
    """Kinetic temperature of a Langevin chain with m, kT, dt, gamma and the
    LJ sigma, epsilon all off 1: <KE> = 3 N kT / 2 (BAOAB's kinetic error is
    O(dt^2), far below the 4% bound here)."""
    sp = I.make_system(22, 2, 3, output_freq=10, mass=m, kT=kT, dt=0.004, gamma=0.5, lj_sigma=1.1, lj_eps=0.7)
    x0 = I.make_chains(8, sp, 3, min_dist=1.0)
    r = orc.explore(sp, x0, 6000, energy=True)
    ke = r["energy"][:, 150:, 2]                 # discard the first 1500 steps
    T = ke.mean() * 2 / (3 * sp.n_beads)
    assert T == pytest.approx(kT, rel=0.04)


def test_lj_sigma_and_epsilon_scale_the_pair_energy(orc):
    """Beads 0 and 3 of a 4-bead chain (bonded terms switched off) interact
    through 4 eps ((sig/r)^12 - (sig/r)^6) - U(rc), with rc an absolute
    cutoff: the minimum sits at r = 2^(1/6) sig with U = -eps - U(rc), the
    force vanishes there, and past rc both are exactly zero."""
    sp = I.make_system(4, 1, 5, lj_sigma=1.1, lj_eps=0.7, bond_k=0.0, angle_k=0.0)
    sp.dihedral_k[:] = 0.0
    rmin = 2 ** (1 / 6) * 1.1
    x = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, rmin, 0]], np.float64)
    U, f, terms = orc.ff(sp, x)
    uc = 4 * 0.7 * ((1.1 / 2.5) ** 12 - (1.1 / 2.5) ** 6)
    assert U == pytest.approx(-0.7 - uc, rel=1e-12)
    assert np.abs(f).max() < 1e-9
    # at r = 1.2 sig: U and the radial force from the closed form
    r = 1.2 * 1.1
    x[3] = [0, r, 0]
    U, f, terms = orc.ff(sp, x)
    sr6 = (1.1 / r) ** 6
    assert U == pytest.approx(4 * 0.7 * (sr6 * sr6 - sr6) - uc, rel=1e-12)
    assert f[3, 1] == pytest.approx(24 * 0.7 * (2 * sr6 * sr6 - sr6) / r, rel=1e-12)
    assert f[0, 1] == pytest.approx(-f[3, 1], rel=1e-12)
    x[3] = [0, 2.5001, 0]
    U, f, terms = orc.ff(sp, x)
    assert U == 0.0 and not f.any()
