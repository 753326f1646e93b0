"""GPU parity of the learned-start kernels against the FP64 oracle (oracle/learned.py), and
the effect of the trained network on the SCF.

Tolerances (derived from the arithmetic):
  descriptors: FP32 exp/cos (relative error ~1e-7 each) summed over <= ~200 atoms of
    values <= 1 -> 2e-5 absolute on sums of order 10.
  forward FP32: two 32/128-term FP32 dot products and tanh per layer on O(1) values:
    ~1e-6 relative per layer, 5e-5 absolute on y.
  forward BF16: operands rounded to 8 mantissa bits (relative 2^-9 each) through three
    layers: a few percent of sum_j |w3_j h2_j|.
  gradient: FP32 sums of up to 64 terms per tile and per-block partials added in FP64:
    1e-4 of the largest gradient component.
"""
import numpy as np
import pytest

from helpers import from_slots, small_cluster

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


@pytest.fixture(scope="module")
def kscf():
    from paper_2303_00790_gb300.build import build
    build()
    from paper_2303_00790_gb300 import kscf as mod
    return mod


def random_net(seed):
    from oracle import learned as L
    rng = np.random.default_rng(seed)
    p = L.init_params(seed)
    for k in ("b1", "b2", "b3"):
        p[k] = 0.2 * rng.standard_normal(p[k].shape)
    return p


def test_descriptors_match_oracle(kscf, species):
    from oracle import learned as L
    from oracle.grid import sphere_grid
    pos, z = small_cluster()
    R, h = 9.0, 0.7
    g, H = kscf.build_cluster(pos, z, species, R, h)
    D = kscf.kscf_descriptors(H, pos, z).cpu().numpy()
    lex, _ = g.slots()
    og = sphere_grid(pos[0], R, h)
    ref = L.descriptors(og.points(), pos, z)
    got = from_slots(D, lex, og.n)
    assert np.max(np.abs(got - ref)) < 2e-5 * max(1.0, np.max(np.abs(ref)))
    assert np.all(D[lex < 0] == 0)
    assert np.max(ref[:, :16]) > 0.5 and np.max(ref[:, 16:]) > 0.5      # both species channels used


@pytest.mark.parametrize("n", [37, 128, 1000])
def test_mlp_forward_and_gradient_match_oracle(kscf, n):
    from oracle import learned as L
    rng = np.random.default_rng(n)
    p = random_net(7)
    Draw = rng.uniform(0, 3, (n, 32))
    mu = rng.uniform(0, 1, 32)
    inv_sd = rng.uniform(0.5, 2, 32)
    x = (Draw.astype(np.float32).astype(np.float64) - mu.astype(np.float32)) * inv_sd.astype(np.float32)
    t = rng.standard_normal(n)
    P = torch.tensor(L.pack(p), dtype=torch.float32, device="cuda")
    mu_d = torch.tensor(mu, dtype=torch.float32, device="cuda")
    isd_d = torch.tensor(inv_sd, dtype=torch.float32, device="cuda")
    D_d = torch.tensor(Draw, dtype=torch.float32, device="cuda")
    t_d = torch.tensor(t, dtype=torch.float32, device="cuda")
    y_ref, (_, h1, h2) = L.forward(p, x)
    y = kscf.kscf_mlp_forward(P, mu_d, isd_d, D_d).cpu().numpy()
    assert np.max(np.abs(y - y_ref)) < 5e-5
    yb = kscf.kscf_mlp_forward(P, mu_d, isd_d, D_d, precision=kscf.KSCF_MLP_BF16).cpu().numpy()
    scale = np.abs(h2) @ np.abs(p["w3"]) + 1e-3
    assert np.all(np.abs(yb - y_ref) < 0.05 * scale)
    assert np.max(np.abs(yb - y_ref)) > 0          # really a different precision
    loss_d = torch.zeros(1, dtype=torch.float64, device="cuda")
    g = kscf.kscf_mlp_loss_grad(P, mu_d, isd_d, D_d, t_d, loss=loss_d).cpu().numpy().astype(np.float64)
    loss_ref, g_ref = L.loss_and_grad(p, x, t.astype(np.float32).astype(np.float64))
    assert abs(loss_d.item() - loss_ref) < 1e-5 * loss_ref
    gr = L.pack(g_ref)
    for key, sl in (("W1", slice(0, 4096)), ("b1", slice(4096, 4224)), ("W2", slice(4224, 20608)),
                    ("b2", slice(20608, 20736)), ("w3", slice(20736, 20864)), ("b3", slice(20864, 20865))):
        err = np.max(np.abs(g[sl] - gr[sl]))
        assert err < 1e-4 * np.max(np.abs(gr)) + 1e-7, (key, err, np.max(np.abs(gr[sl])))


def test_adam_matches_oracle(kscf):
    from oracle import learned as L
    rng = np.random.default_rng(2)
    flat = rng.standard_normal(L.N_PARAMS)
    P = torch.tensor(flat, dtype=torch.float32, device="cuda")
    m = torch.zeros_like(P)
    v = torch.zeros_like(P)
    params = {"a": flat.astype(np.float32).astype(np.float64)}
    mm = {"a": np.zeros(L.N_PARAMS)}
    vv = {"a": np.zeros(L.N_PARAMS)}
    for step in range(1, 4):
        gnp = rng.standard_normal(L.N_PARAMS).astype(np.float32)
        kscf.kscf_mlp_adam(P, torch.tensor(gnp, device="cuda"), m, v, step, 1e-2)
        params, mm, vv = L.adam_step(params, {"a": gnp.astype(np.float64)}, mm, vv, step, 1e-2)
    assert np.max(np.abs(P.cpu().numpy() - params["a"])) < 1e-6


def test_standardize_matches_oracle(kscf):
    """FP64 sums of FP32 inputs: mu, inv_sd and the target statistics to ~1e-12 relative
    before the rounding of the stored FP32 values (half an ulp, 6e-8)."""
    from oracle import learned as L
    rng = np.random.default_rng(12)
    n = 10007
    D = rng.uniform(0, 3, (n, 32)).astype(np.float32)
    D[:, 11] = 0.5                       # constant feature: switched off
    t = (0.2 * rng.standard_normal(n) - 0.05).astype(np.float32)
    mu, isd, tn, ts, sc = kscf.kscf_mlp_standardize(torch.tensor(D, device="cuda"), torch.tensor(t, device="cuda"))
    rmu, risd, rts, rsc, rtn = L.standardise(D.astype(np.float64), t.astype(np.float64))
    assert np.allclose(mu.cpu().numpy(), rmu, rtol=1e-7, atol=0)
    assert np.allclose(isd.cpu().numpy(), risd, rtol=1e-7, atol=0) and isd[11].item() == 0.0
    assert abs(ts - rts) < 1e-12 * abs(rsc) and abs(sc - rsc) < 1e-12 * rsc
    assert np.allclose(tn.cpu().numpy(), rtn, rtol=0, atol=1e-6)


def test_correction_and_training_data_match_oracle(kscf, species):
    """kscf_mlp_correction = the oracle's de-standardised network (FP32 forward tolerance
    times t_scale); kscf_mlp_training_data = descriptors and V_in - V_start of the domain
    points, in lexicographic order."""
    from oracle import learned as L
    p = random_net(8)
    rng = np.random.default_rng(2)
    D = rng.uniform(0, 2, (777, 32))
    mu, isd = D.mean(0), 1.0 / D.std(0)
    P = torch.tensor(L.pack(p), dtype=torch.float32, device="cuda")
    dv = kscf.kscf_mlp_correction(P, torch.tensor(mu, dtype=torch.float32, device="cuda"),
                                  torch.tensor(isd, dtype=torch.float32, device="cuda"), 0.37, 2.5,
                                  torch.tensor(D, dtype=torch.float32, device="cuda"))
    ref = L.correction(p, mu.astype(np.float32).astype(np.float64), isd.astype(np.float32).astype(np.float64),
                       0.37, 2.5, D.astype(np.float32).astype(np.float64))
    assert dv.dtype == torch.float64 and np.max(np.abs(dv.cpu().numpy() - ref)) < 5e-5 * 2.5
    # training data of a (not yet self-consistent) SCF state: the definition on the host
    pos, z = small_cluster()
    g, H = kscf.build_cluster(pos, z, species, 9.0, 0.7)
    S = kscf.Scf(H, pos, z, species, kscf.scf_params(8, 8))
    S.start(seed=1)
    S.step()
    Ds = kscf.kscf_descriptors(H, pos, z)
    Dp, tp = kscf.kscf_mlp_training_data(S, Ds, g.info["n_points"])
    torch.cuda.synchronize()
    lex, _ = g.slots()
    n = g.info["n_points"]
    want_t = L.training_target(from_slots(S.get(kscf.KSCF_FIELD_V_IN).cpu().numpy(), lex, n),
                               from_slots(S.get(kscf.KSCF_FIELD_V_START).cpu().numpy(), lex, n))
    assert np.array_equal(Dp.cpu().numpy(), from_slots(Ds.cpu().numpy(), lex, n))
    assert np.array_equal(tp.cpu().numpy(), want_t.astype(np.float32))
    S.free()


def test_training_fits_a_smooth_target(kscf):
    from paper_2303_00790_gb300 import learned
    rng = np.random.default_rng(0)
    D = torch.tensor(rng.uniform(0, 2, (20000, 32)), dtype=torch.float32, device="cuda")
    T = torch.sin(D[:, 0] * 2.0) + 0.5 * D[:, 5] * D[:, 17]
    model, losses = learned.train(D, T, steps=600, batch=4096, lr=3e-3, log_every=100)
    # standardised target: the initial loss is ~1; the fit explains > 99 % of the variance
    assert losses[-1][1] < 0.01, losses
    pred = kscf.kscf_mlp_correction(model.params, model.mu, model.inv_sd, model.t_shift, model.t_scale, D)
    r2 = 1.0 - torch.mean((pred - T) ** 2).item() / torch.var(T).item()
    assert r2 > 0.99, r2


def test_learned_start_reduces_scf_steps(kscf, species):
    from paper_2303_00790_gb300 import learned
    from workloads.cluster import cluster_for_diameter, random_rotation, training_clusters
    from workloads.configs import cluster_scf_config
    Ds, Ts = [], []
    for seed, d, pos, z in training_clusters(8, seed0=2000, d_min_nm=1.0, d_max_nm=1.7):
        D, T, info = learned.sample_cluster(pos, z, species, cluster_scf_config(d, z))
        assert info["converged"], (seed, d)
        Ds.append(D)
        Ts.append(T)
    model, losses = learned.train(torch.cat(Ds), torch.cat(Ts), steps=1500, batch=16384, lr=2e-3, log_every=500)
    d = 1.9
    pos, z = cluster_for_diameter(d)
    pos = pos @ random_rotation(4242).T
    cfg = cluster_scf_config(d, z)
    base, _, exb = learned.run_scf(pos, z, species, cfg)
    lrn, _, exl = learned.run_scf(pos, z, species, cfg, dv=lambda H: model.correction(H, pos, z))
    assert base[-1]["converged"] and lrn[-1]["converged"]
    # the same fixed point: energies agree within the SCF tolerance's reach
    e_ref = exb["final"]["e_total"]
    assert abs(exl["final"]["e_total"] - e_ref) < 1e-6 * len(z)
    # the learned start reaches the converged energy (1e-6 Ha/atom) and self-consistency sooner
    e_last = base[-1]["e_total"]          # per-step energies share the in-loop evaluation
    n_b = learned.steps_to_energy(base, e_last, len(z))
    n_l = learned.steps_to_energy(lrn, e_last, len(z))
    print(f"learned start: first SRE {lrn[0]['sre_ry']:.1f} vs {base[0]['sre_ry']:.1f} Ry, steps {len(lrn)} vs "
          f"{len(base)}, steps to 1e-6 Ha/atom {n_l} vs {n_b}")
    # the gain: a much better starting potential, fewer SCF steps to the converged energy
    # and to self-consistency
    assert lrn[0]["sre_ry"] < 0.6 * base[0]["sre_ry"], (lrn[0]["sre_ry"], base[0]["sre_ry"])
    assert n_l < n_b and len(lrn) < len(base), (n_l, n_b, len(lrn), len(base))
