"""Learned surrogate of the intralaminar law (include/pdn_surrogate.h).

* The GPU gradient (BF16 tensor-core products, FP32 sums) equals FP64
  backpropagation with the same BF16 rounding points (tests/mlp_reference.py,
  itself pinned by finite differences) to FP32 round-off, and plain FP64
  backpropagation to the BF16 precision.
* The exact law that generates the training data equals the FP64 oracle's
  point law.
* Generated points lie in the surrogate's regime (no threshold grows).
"""
import numpy as np
import pytest

import mlp_reference as R
import oracle
import pdn_inputs as pi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_2301_05552_gb300 as p
    p.lib()
    return p


def _mat():
    return pi.material_im7_like_config(t_ply=0.275, spread=0.0)


LC = 0.552  # crack-band length of the 128x192x16 plate's elements (mm)


def _blocks(g):
    out, o = [], 0
    for s in R.SHAPES:
        n = int(np.prod(s))
        out.append(g[o:o + n])
        o += n
    return out


def test_gradient_matches_fp64_backprop(pkg):
    s = pkg.pdn_sur_create(_mat(), LC, seed=7)
    p, _ = pkg.pdn_sur_get_params(s)
    rng = np.random.default_rng(1)
    n = 256
    xn = rng.normal(size=(n, 10)).astype(np.float32)
    tn = rng.normal(size=(n, 10)).astype(np.float32)
    g, loss = pkg.pdn_sur_gradient(s, xn, tn)
    p64 = p.astype(np.float64)
    lb, gb = R.loss_and_grad(p64, xn.astype(np.float64), tn.astype(np.float64), bf=True)
    l64, g64 = R.loss_and_grad(p64, xn.astype(np.float64), tn.astype(np.float64), bf=False)
    assert abs(loss - lb) <= 1e-5 * lb
    assert abs(loss - l64) <= 2e-2 * l64
    for gg, rb, r64 in zip(_blocks(g.astype(np.float64)), _blocks(gb), _blocks(g64)):
        nb = np.linalg.norm(rb)
        assert np.linalg.norm(gg - rb) <= 2e-3 * nb + 1e-12
        assert np.linalg.norm(gg - r64) <= 5e-2 * np.linalg.norm(r64) + 1e-12
    # the parameters did not move
    p2, _ = pkg.pdn_sur_get_params(s)
    assert np.array_equal(p, p2)
    s.close()


def test_tensor_core_forward_matches_fp64_reference(pkg):
    """Inference on the Blackwell tensor cores (tcgen05, TMEM accumulators,
    128 points per CTA; 1,000 points leave a partial last CTA) against the
    FP64 forward pass with the same bf16 rounding points, and against plain
    FP64 to the bf16 precision, for the initial and a perturbed network."""
    s = pkg.pdn_sur_create(_mat(), LC, seed=7)
    p, sc = pkg.pdn_sur_get_params(s)
    rng = np.random.default_rng(4)
    for trial in range(2):
        if trial == 1:
            p = (p + rng.normal(scale=0.05, size=p.shape)).astype(np.float32)
            pkg.pdn_sur_set_params(s, p, sc)
        x = rng.normal(size=(1000, 10)).astype(np.float32)
        y = pkg.pdn_sur_forward(s, x).astype(np.float64)
        xn = (x.astype(np.float64) - sc[0:10]) * sc[10:20]
        yb = R.forward_bf16(p.astype(np.float64), xn) * sc[30:40] + sc[20:30]
        y64 = R.forward(p.astype(np.float64), xn) * sc[30:40] + sc[20:30]
        scale = np.abs(yb).max()
        assert np.abs(y - yb).max() <= 1e-2 * scale
        assert np.sqrt(np.mean((y - yb) ** 2)) <= 1e-3 * scale
        assert np.abs(y - y64).max() <= 5e-2 * scale
    s.close()


def test_exact_law_matches_oracle_point_law(pkg):
    s = pkg.pdn_sur_create(_mat(), LC, seed=0)
    rng = np.random.default_rng(2)
    n = 400
    x = np.zeros((n, 10), dtype=np.float32)
    x[:, :3] = rng.uniform(-0.02, 0.02, size=(n, 3))
    x[:, 3:6] = rng.uniform(-0.04, 0.04, size=(n, 3))
    x[:, 6:] = np.where(rng.uniform(size=(n, 4)) < 0.5, 1.0, rng.uniform(1.0, 3.0, size=(n, 4)))
    y = pkg.pdn_sur_exact(s, x)
    mat = _mat()
    for i in range(n):
        h = np.array([*x[i, 6:].astype(np.float64), 0.0, 0.0, 0.0])
        sig, ho = oracle.cdm_point(mat, LC, x[i, :6].astype(np.float64), h, damage_on=True, plasticity_on=False)
        scale = max(np.abs(sig).max(), 1.0)
        assert np.abs(y[i, :6] - sig).max() <= 1e-5 * scale, i
        assert np.allclose(y[i, 6:], ho[:4], rtol=1e-6), i
    s.close()


def test_generated_points_are_in_the_regime_and_deterministic(pkg):
    s1 = pkg.pdn_sur_create(_mat(), LC)
    s2 = pkg.pdn_sur_create(_mat(), LC)
    n1 = pkg.pdn_sur_generate(s1, 3000, 8, 0.01, 0.4, 0.9, seed=5)
    n2 = pkg.pdn_sur_generate(s2, 3000, 8, 0.01, 0.4, 0.9, seed=5)
    assert n1 == n2 and 0.2 * 3000 * 8 < n1 <= 3000 * 8
    x1, y1 = pkg.pdn_sur_get_data(s1, 0, n1)
    x2, y2 = pkg.pdn_sur_get_data(s2, 0, n1)
    assert np.array_equal(x1, x2) and np.array_equal(y1, y2)
    # no threshold grows in the regime, and thresholds start at 1
    assert np.array_equal(x1[:, 6:], y1[:, 6:])
    assert (x1[:, 6:] >= 1.0).all()
    # some kept points are damaged (thresholds above 1: unloading after onset)
    assert (x1[:, 6:] > 1.0).any()
    # the exact law reproduces the stored targets
    yy = pkg.pdn_sur_exact(s1, x1[:2000])
    assert np.allclose(yy, y1[:2000], rtol=1e-6, atol=1e-6)
    s1.close()
    s2.close()


def test_set_surrogate_rejects_unsupported_contexts(pkg):
    w = pi.plain_fp64_plate(nx=8, ny=8)
    g = pkg.Solver(w)  # FP64 element mode
    s = pkg.pdn_sur_create(_mat(), LC)
    with pytest.raises(pkg.PdnError) as e:
        pkg.pdn_set_surrogate(g.ctx, s, 0.9)
    assert e.value.code == -1
    pkg.pdn_set_surrogate(g.ctx, None)  # back to the exact law is always allowed
    s.close()
    g.close()


@pytest.fixture(scope="module")
def trained(pkg):
    """A surrogate trained on 300k paths for 10,000 Adam steps (about 1.5 s)."""
    s = pkg.pdn_sur_create(_mat(), LC, seed=1)
    n = pkg.pdn_sur_generate(s, 300_000, 8, 0.01, 0.4, 0.9, seed=11)
    loss = pkg.pdn_sur_train(s, 10_000, 8192, 2e-3, seed=3)
    yield s, n, loss
    s.close()


def test_training_fits_held_out_points(pkg, trained):
    """Held-out points of other paths (another seed): stress within a few
    percent of the exact law (RMS, relative to each component's RMS), the
    thresholds (unchanged in the regime) within 0.1."""
    s, n, loss = trained
    assert n > 1_000_000
    assert loss[-1] < loss[0] / 300.0
    h = pkg.pdn_sur_create(_mat(), LC, seed=0)
    nh = pkg.pdn_sur_generate(h, 5000, 8, 0.01, 0.4, 0.9, seed=99)
    x, y = pkg.pdn_sur_get_data(h, 0, nh)
    h.close()
    yp = pkg.pdn_sur_forward(s, x)
    rms = np.sqrt(np.mean(y[:, :6].astype(np.float64) ** 2, axis=0))
    rel = np.sqrt(np.mean((yp[:, :6] - y[:, :6]).astype(np.float64) ** 2, axis=0)) / rms
    assert (rel < 0.04).all(), rel
    assert np.max(np.abs(yp[:, 6:] - y[:, 6:])) < 0.1


def test_impact_with_learned_law(pkg, trained):
    """The reduced damage plate of the FP32 parity test with the learned law
    where it applies: the peak contact force stays within 0.5 % of the exact
    law's, and the run can return to the exact law."""
    s, _, _ = trained
    w = pi.damage_fp32_plate(nx=32, ny=48, Lx=25.0, Ly=37.5, H=4.4, mass=5.5e-3 / 16, steps=3000)
    ge = pkg.Solver(w, precision=pkg.PDN_FP32_FORCE)
    ge.step(3000)
    gl = pkg.Solver(w, precision=pkg.PDN_FP32_FORCE)
    pkg.pdn_set_surrogate(gl.ctx, s, 0.9)
    gl.step(2000)
    pkg.pdn_set_surrogate(gl.ctx, None)
    gl.step(1000)
    fe, fl = ge.force_history(), gl.force_history()
    assert fe.max() > 0.0
    assert abs(fl.max() - fe.max()) <= 5e-3 * fe.max()
    de = ge.state()[0]
    dl = gl.state()[0]
    assert np.abs(dl - de).max() <= 5e-2 * np.abs(de).max()
    ge.close()
    gl.close()


def test_learned_law_impact_against_the_oracle(pkg, trained):
    """The whole impact run with the learned law where it applies (the exact
    law elsewhere), judged against the FP64 oracle's exact law on the
    reduced damage plate: peak contact force within 0.5 % of the oracle's
    and the force history within 1 % of its peak at every step."""
    s, _, _ = trained
    w = pi.damage_fp32_plate(nx=32, ny=48, Lx=25.0, Ly=37.5, H=4.4, mass=5.5e-3 / 16, steps=3000)
    gl = pkg.Solver(w, precision=pkg.PDN_FP32_FORCE)
    pkg.pdn_set_surrogate(gl.ctx, s, 0.9)
    o = oracle.model_for(w)
    for _ in range(30):
        gl.step(100)
        assert o.step(100) == 0
    fl, fo = gl.force_history(), o.force_history()
    assert len(fl) == len(fo) == 3000 and fo.max() > 0.0
    pk = abs(fl.max() - fo.max()) / fo.max()
    hist_err = float(np.abs(fl - fo).max() / fo.max())
    print(f"\nlearned law vs FP64 oracle: peak {fl.max():.3f} vs {fo.max():.3f} N (rel {pk:.2e}), "
          f"history err {hist_err:.2e} of peak")
    assert pk <= 5e-3
    assert hist_err <= 1e-2
    gl.close()
    o.close()


def test_empty_training_box_falls_back_to_the_exact_law(pkg, trained):
    """With a training box that contains no point every Gauss point takes the
    exact law: the run follows the exact-law run to FP32 rounding (the two
    hex kernels evaluate the same formulas in a different order)."""
    s, _, _ = trained
    p, sc = pkg.pdn_sur_get_params(s)
    s2 = pkg.pdn_sur_create(_mat(), LC)
    sc2 = sc.copy()
    sc2[40:50] = 1e30   # lo
    sc2[50:60] = -1e30  # hi
    pkg.pdn_sur_set_params(s2, p, sc2)
    w = pi.damage_fp32_plate(nx=32, ny=48, Lx=25.0, Ly=37.5, H=4.4, mass=5.5e-3 / 16, steps=1500)
    ge = pkg.Solver(w, precision=pkg.PDN_FP32_FORCE)
    gl = pkg.Solver(w, precision=pkg.PDN_FP32_FORCE)
    pkg.pdn_set_surrogate(gl.ctx, s2, 0.9)
    ge.step(1500)
    gl.step(1500)
    de, dl = ge.state()[0], gl.state()[0]
    assert np.abs(dl - de).max() <= 1e-4 * np.abs(de).max()
    fe, fl = ge.force_history(), gl.force_history()
    assert fe.max() > 0.0 and abs(fl.max() - fe.max()) <= 1e-4 * fe.max()
    s2.close()
    ge.close()
    gl.close()


def test_learned_law_local_repeat_equals_full_repeat(pkg, trained, monkeypatch):
    """The hex kernel of the learned law evaluates, in a repeated pass, only
    the elements of released nodes (its warps still run together); a run
    with PDN_FULL_REPEAT=1 (every element again) is bitwise the same."""
    s, _, _ = trained
    w = pi.damage_fp32_plate(nx=32, ny=48, Lx=25.0, Ly=37.5, H=4.4, mass=5.5e-3 / 16, steps=3000)
    runs = []
    for full in ("0", "1"):
        monkeypatch.setenv("PDN_FULL_REPEAT", full)
        g = pkg.Solver(w, precision=pkg.PDN_FP32_FORCE)
        pkg.pdn_set_surrogate(g.ctx, s, 0.9)
        g.step(2500)
        d, v, _ = g.state()
        runs.append((d, v, g.force_history(), pkg.pdn_damage_field(g.ctx, "D2"), g.info()["n_repeats"]))
        g.close()
    (d0, v0, f0, k0, r0), (d1, v1, f1, k1, r1) = runs
    assert r0 == r1
    assert np.array_equal(d0, d1) and np.array_equal(v0, v1)
    assert np.array_equal(f0, f1) and np.array_equal(k0, k1)
