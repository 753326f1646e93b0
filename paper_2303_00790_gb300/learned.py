"""Learned SCF start: data from converged SCF runs, training with the library's MLP
kernels on the GPU, and the predicted correction of the superposition starting potential.

Host orchestration only (which clusters, which batches, when to stop); the descriptors,
the training targets, the standardisation, the network's forward and backward passes,
the de-standardised correction, the optimiser and every SCF step run in libkscf's
kernels through the C ABI.  The target of the network is
    dV = V_in(converged) - V_start(superposition of neutral atoms)
on the domain points, standardised by its mean and standard deviation; the inputs are
the 32 radial descriptors standardised per feature over the training set.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass

import numpy as np

from . import kscf


def glorot_params(seed: int) -> np.ndarray:
    """Initial parameter vector: Glorot-uniform weights, zero biases (seeded)."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_in, fan_out in ((32, 128), (128, 128), (128, 1)):
        lim = math.sqrt(6.0 / (fan_in + fan_out))
        parts.append(rng.uniform(-lim, lim, fan_in * fan_out))
        parts.append(np.zeros(fan_out))
    flat = np.concatenate(parts).astype(np.float32)
    assert flat.size == kscf.KSCF_MLP_N_PARAMS
    return flat


@dataclass
class LearnedStart:
    params: "object"      # torch float32 (N_PARAMS,) on the device
    mu: "object"          # torch float32 (32,)
    inv_sd: "object"      # torch float32 (32,)
    t_shift: float
    t_scale: float

    def correction(self, ham, atom_pos, atom_z, precision: int = kscf.KSCF_MLP_BF16):
        """dV per slot (torch float64, device) for kscf_scf_start."""
        D = kscf.kscf_descriptors(ham, atom_pos, atom_z)
        return kscf.kscf_mlp_correction(self.params, self.mu, self.inv_sd, self.t_shift, self.t_scale, D, precision)

    def state(self) -> dict:
        return {"params": self.params.cpu().numpy(), "mu": self.mu.cpu().numpy(),
                "inv_sd": self.inv_sd.cpu().numpy(), "t_shift": self.t_shift, "t_scale": self.t_scale}

    @staticmethod
    def from_state(st: dict) -> "LearnedStart":
        import torch
        dev = "cuda"
        return LearnedStart(torch.tensor(st["params"], device=dev), torch.tensor(st["mu"], device=dev),
                            torch.tensor(st["inv_sd"], device=dev), float(st["t_shift"]), float(st["t_scale"]))


# Settings of the learned-start runs.  Electronic temperature (Ha): small enough to
# leave closed shells untouched (gaps of the synthetic clusters are >= ~0.01 Ha), large
# enough to let clusters whose highest level is a partly filled degenerate one converge.
# Anderson step 0.5 with the Kerker preconditioner (q0 = 0.5 / bohr): the best of the
# settings compared on 2.0-2.4 nm clusters (some of which oscillate with plain Anderson
# mixing at steps above ~0.1).
KT_DEFAULT = 1e-3
ALPHA_DEFAULT = 0.5
KERKER_DEFAULT = 0.5
E_TOL_PER_ATOM = 1e-6


def scf_until(S, n_atoms: int, max_steps: int, e_tol_per_atom: float = 0.0, settle: int = 3):
    """Steps the SCF until it converges (SRE below the handle's tolerance) or, when
    e_tol_per_atom > 0, until the total energy has changed by less than e_tol_per_atom * n_atoms
    over `settle` consecutive steps; at most max_steps steps."""
    reps = []
    quiet = 0
    for _ in range(max_steps):
        r = S.step()
        reps.append(r)
        if r["converged"]:
            break
        if e_tol_per_atom > 0 and len(reps) > 1:
            quiet = quiet + 1 if abs(reps[-1]["e_total"] - reps[-2]["e_total"]) < e_tol_per_atom * n_atoms else 0
            if quiet >= settle:
                break
    return reps


def run_scf(pos, z, species, cfg: dict, dv=None, seed: int = 1, max_steps: int = 100, dtype=None, mode=None,
            keep=False, kT: float = KT_DEFAULT, alpha: float = ALPHA_DEFAULT, e_tol_per_atom: float = 0.0,
            kerker_q0: float = KERKER_DEFAULT, first_iters: int = 4):
    """SCF on one cluster (mixed precision by default).  Returns (reports, wall_s, extra)
    where extra holds the grid/Hamiltonian/handle when keep=True."""
    import torch
    dtype = kscf.KSCF_F32 if dtype is None else dtype
    mode = (kscf.KSCF_GEMM_TENSOR if dtype == kscf.KSCF_F32 else kscf.KSCF_GEMM_NATIVE) if mode is None else mode
    g, H = kscf.build_cluster(pos, z, species, cfg["radius"], cfg["h"])
    params = kscf.scf_params(cfg["k"], cfg["degree"], dtype=dtype, gemm_mode=mode, kT=kT, mix_alpha=alpha,
                             kerker_q0=kerker_q0, first_iters=first_iters)
    S = kscf.Scf(H, pos, z, species, params)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    dv_t = dv(H) if callable(dv) else dv
    S.start(seed=seed, dv_start=dv_t)
    reps = scf_until(S, len(z), max_steps, e_tol_per_atom)
    ev = S.evaluate()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    extra = {"grid": g, "ham": H, "scf": S, "final": ev}
    if not keep:
        S.free()
        extra = {"final": ev}
    return reps, wall, extra


# a training potential is accepted when its SRE is below this (Ry): the residual
# potential is then ~1e-4 Ha RMS, far below what the network resolves
SRE_ACCEPT_RY = 2e-3


def sample_cluster(pos, z, species, cfg: dict, seed: int = 1, **scf_kw):
    """(D, dV, info) of the domain points of one self-consistent cluster (float32 device
    tensors); (None, None, info) when its SCF does not reach SRE < SRE_ACCEPT_RY in 100
    steps."""
    import torch
    reps, wall, ex = run_scf(pos, z, species, cfg, seed=seed, keep=True, **scf_kw)
    if not (reps[-1]["converged"] or reps[-1]["sre_ry"] < SRE_ACCEPT_RY):
        ex["scf"].free()
        return None, None, {"steps": len(reps), "wall_s": wall, "converged": False}
    g, H, S = ex["grid"], ex["ham"], ex["scf"]
    D, t = kscf.kscf_mlp_training_data(S, kscf.kscf_descriptors(H, pos, z), g.info["n_points"])
    torch.cuda.synchronize()
    S.free()
    return D, t, {"steps": len(reps), "wall_s": wall, "converged": True, "sre_ry": reps[-1]["sre_ry"]}


def train(D, T, steps: int = 3000, batch: int = 16384, lr: float = 2e-3, seed: int = 0, log_every: int = 0):
    """Fits the network to (D, T) (device float32; T raw dV) with Adam on random batches.
    Returns (LearnedStart, losses)."""
    import torch
    mu, inv_sd, Tn, t_shift, t_scale = kscf.kscf_mlp_standardize(D, T)
    P = torch.tensor(glorot_params(seed), device="cuda")
    m = torch.zeros_like(P)
    v = torch.zeros_like(P)
    g = torch.empty_like(P)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    n = D.shape[0]
    b = min(batch, n)
    work = torch.empty(kscf.kscf_mlp_work_size(b), dtype=torch.uint8, device="cuda")
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    losses = []
    Db = torch.empty((b, D.shape[1]), dtype=torch.float32, device="cuda")
    Tb = torch.empty(b, dtype=torch.float32, device="cuda")
    for it in range(1, steps + 1):
        idx = torch.randint(0, n, (b,), device="cuda", generator=gen)
        torch.index_select(D, 0, idx, out=Db)
        torch.index_select(Tn, 0, idx, out=Tb)
        kscf.kscf_mlp_loss_grad(P, mu, inv_sd, Db, Tb, grad=g, loss=loss, work=work)
        # cosine decay of the step size over the run
        lr_t = lr * 0.5 * (1.0 + math.cos(math.pi * (it - 1) / steps))
        kscf.kscf_mlp_adam(P, g, m, v, it, max(lr_t, 1e-6))
        if log_every and (it % log_every == 0 or it == steps):
            losses.append((it, float(loss.item())))
    return LearnedStart(P, mu, inv_sd, t_shift, t_scale), losses


def steps_to_energy(reports, e_ref: float, n_atoms: int, tol_per_atom: float = 1e-6) -> int:
    """First SCF step after which |E - e_ref| stays below tol * n_atoms (len+1 if never)."""
    ok = [abs(r["e_total"] - e_ref) < tol_per_atom * n_atoms for r in reports]
    for i in range(len(ok)):
        if all(ok[i:]):
            return i + 1
    return len(reports) + 1
