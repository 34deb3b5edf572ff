"""Builds the oracle mesh and the GPU context from one workload description."""
import numpy as np

from paper_2409_10383_gb300 import inputs

NF = 22
PARAM_KEYS = ("lapse", "shift", "ko_sigma", "kappa1", "kappa2", "eta", "chi_floor")


def oracle_mesh(oracle, w):
    return oracle.Mesh(n=w["n"], lo=w["lo"], h=w["h"], ghosts=w["ghosts"], order=w["order"],
                       dom_lo=w["dom_lo"], dom_hi=w["dom_hi"], periodic=w["periodic"],
                       level=w.get("level"), **{k: w[k] for k in PARAM_KEYS})


def gpu_ctx(w, precision=64, schedule=0):
    from paper_2409_10383_gb300.z4c import Z4c
    return Z4c.from_workload(w, precision=precision, schedule=schedule)


def small_workload(kind, order, nb=(1, 1, 1), n=16, periodic=None, **over):
    """A small mesh with the physics of one of the paper's problems."""
    if kind == "gauge_wave":
        w = dict(ghosts=order // 2 + 1, order=order, periodic=True, dom_lo=(-0.5,) * 3,
                 dom_hi=(0.5,) * 3, lapse=0, shift=0, ko_sigma=0.02, kappa1=0.0, kappa2=0.0,
                 eta=0.0, chi_floor=1e-6, id_kind=inputs.ID_GAUGE_WAVE, id_par=[0.01, 1.0, 0.0])
    else:
        w = dict(ghosts=order // 2 + 1, order=order, periodic=False, dom_lo=(-4.0,) * 3,
                 dom_hi=(4.0,) * 3, lapse=1, shift=1, ko_sigma=0.5, kappa1=0.02, kappa2=0.0,
                 eta=2.0, chi_floor=1e-6, id_kind=inputs.ID_SCHWARZSCHILD, id_par=[1.0, 0.0])
    if periodic is not None:
        w["periodic"] = periodic
    w.update(over)
    n3 = np.array((n, n, n) if np.isscalar(n) else tuple(n))
    # spacing from the x extent; the box is centred on the origin
    h = (w["dom_hi"][0] - w["dom_lo"][0]) / (nb[0] * n3[0])
    half = np.array(nb) * n3 * h / 2
    w["dom_lo"], w["dom_hi"] = tuple(-half), tuple(half)
    w["n"], w["lo"], w["h"] = inputs.uniform_blocks(nb, tuple(n3), w["dom_lo"], w["dom_hi"])
    return w


def field_errors(oracle_mesh_, ref, got, mask_fn="evolved"):
    """err_f = max|got - ref| / D_f over evolved (or interior) cells, with
    D_f = max(||ref_f||_inf, 1e-3 max_g ||ref_g||_inf)."""
    m = oracle_mesh_
    R, G = [], []
    for b in range(m.nblocks):
        mk = m.evolved_mask(b) if mask_fn == "evolved" else m.interior_mask(b)
        R.append(m.blocks(ref)[b][:, mk])
        G.append(m.blocks(got)[b][:, mk])
    R = np.concatenate(R, axis=1)
    G = np.concatenate(G, axis=1)
    scale = np.abs(R).max(axis=1)
    D = np.maximum(scale, 1e-3 * scale.max())
    D[D == 0] = 1.0
    return np.abs(G - R).max(axis=1) / D, np.abs(G - R).max(axis=1)


def perturb(m, u, seed, amp):
    for blk, p in zip(m.blocks(u), inputs.perturbation([m.ext(b)[::-1] for b in range(m.nblocks)],
                                                       seed, amp)):
        blk += p
    return u
