"""Helpers shared by the parity tests: oracle set-up from a seeded world, per-channel error
metric, and the decision band (cells whose float decisions were near-ties in the oracle)."""
import numpy as np

from oracle import coral_oracle as O

FP32_TOL = 1e-5        # per-channel normwise relative error, FP32 path
BF16_TOL = 2e-2        # per-channel normwise relative error, BF16 path vs the FP64 oracle
FP32_TAU = 1e-4        # decision band, FP32 path
BF16_TAU = 3e-2        # decision band, BF16 path vs the FP64 oracle


def oracle_setup(world, **pkw):
    st = O.State.from_world(world)
    p = O.Params.from_world(world, **pkw)
    gen = None
    if world.genes is not None:
        gen = O.Genomes.from_genes(world.genes, world.capacity)
        nets = O.nets_from_genomes(gen, world.hidden)
    else:
        nets = O.Nets.from_dense(world.dense, world.hidden, world.capacity)
    return st, nets, gen, p


def round32(st: O.State) -> O.State:
    """The state as float32 storage holds it (what the GPU is loaded with)."""
    f = lambda a: a.astype(np.float32).astype(np.float64)
    return O.State(st.width, st.height, f(st.E), f(st.I), f(st.C), st.G.copy(), st.R.copy())


def state_arrays(st: O.State):
    H, W = st.height, st.width
    return (st.E.reshape(H, W).astype(np.float32), st.I.reshape(H, W).astype(np.float32),
            st.C.reshape(4, H, W).astype(np.float32), st.G.reshape(H, W).astype(np.int32),
            st.R.reshape(H, W).astype(np.uint8))


def rel_err(gpu, ora, mask=None):
    """[R16] max |gpu - ora| / max(max |ora|, 1e-30) over the (unmasked) cells of a plane."""
    g = np.asarray(gpu, np.float64).ravel()
    o = np.asarray(ora, np.float64).ravel()
    if mask is not None:
        g, o = g[~mask], o[~mask]
    if o.size == 0:
        return 0.0
    return float(np.max(np.abs(g - o)) / max(float(np.max(np.abs(o))), 1e-30))


def explore_band(st: O.State, z, margin, tau, rotation=1):
    """Cells whose incoming exploration may legitimately differ because an explorer's decision
    was within tau of flipping (z, margin: full-length pass-1 pre-activations and explore
    margins of the oracle, NaN where not computed): every such explorer and the targets of
    each of its explore actuators within tau of the maximum (one of them may be picked
    instead, or none when the maximum is within tau of zero)."""
    W, H = st.width, st.height
    ex = np.nan_to_num(margin, nan=np.inf) < tau
    m = ex.copy()
    idx = np.nonzero(ex)[0]
    if idx.size:
        zl = z[idx, 6:10]
        top = zl.max(axis=1)
        Rv = st.R[idx] if rotation else np.zeros(idx.size, np.int64)
        for k in range(4):
            cand = zl[:, k] >= top - tau
            d = (Rv[cand] + O.EXPLORE_TURN[k]) % 4
            for D, (dx, dy) in enumerate(O.DIRS):
                sel = idx[cand][d == D]
                m[O.neighbour(W, H, sel, dx, dy)] = True
    return m


def band_mask(st: O.State, info, tau, rotation=1):
    """Cells whose I, G or R may legitimately differ because a float decision of the oracle
    was within tau of flipping: explorers in band and their candidate targets, and target
    cells whose winner or takeover compare was in band."""
    return explore_band(st, info["z"], info["margin_explore"], tau, rotation) | (info["margin_target"] < tau)


def band_mask_cells(st: O.State, o, cells, tau, rotation=1):
    """band_mask for the listed cells of ``O.step_cells`` output ``o``."""
    p1 = o["pass1"]
    return explore_band(st, p1["z"], p1["margin"], tau, rotation)[np.asarray(cells)] | (o["tmargin"] < tau)


def decision_split(st: O.State, dir_a, dir_b, G_a, G_b, R_a, R_b, rotation=1):
    """Cells whose I, G or R follow a decision that two oracle variants (e.g. the FP64 network
    and the BF16-operand network) take differently: explorers whose direction differs and their
    targets under either direction, and cells whose takeover outcome (G, R) differs.
    dir_*: full-length pass-1 directions (-1 none, -2 not computed); G_*, R_*: next states,
    full length or at the listed cells (then the explorer part is returned full length too)."""
    W, H = st.width, st.height
    ok = (dir_a > -2) & (dir_b > -2)
    dd = ok & (dir_a != dir_b)
    m = dd.copy()
    for d in (dir_a, dir_b):
        idx = np.nonzero(dd & (d >= 0))[0]
        for D, (dx, dy) in enumerate(O.DIRS):
            m[O.neighbour(W, H, idx[d[idx] == D], dx, dy)] = True
    return m, (np.asarray(G_a) != np.asarray(G_b)) | (np.asarray(R_a) != np.asarray(R_b))


def band_breakdown(st: O.State, info, tau, rotation=1):
    """Fractions of cells: in the band, explorers within tau, target compares within tau."""
    ex = info["margin_explore"] < tau
    tg = info["margin_target"] < tau
    return {"band": float(band_mask(st, info, tau, rotation).mean()), "explore_margin": float(ex.mean()),
            "target_margin": float(tg.mean())}


def compare_step(gpu, new: O.State, mask, tol):
    """Per-channel errors (dict) and integer mismatches outside the mask."""
    H, W = new.height, new.width
    errs = {"E": rel_err(gpu["E"], new.E), "I": rel_err(gpu["I"], new.I, mask)}
    for k in range(4):
        errs[f"C{k}"] = rel_err(gpu["C"][k], new.C[k])
    gG = gpu["G"].ravel().astype(np.int64)
    gR = gpu["R"].ravel().astype(np.int64)
    bad_G = int(np.sum((gG != new.G) & ~mask))
    bad_R = int(np.sum((gR != new.R) & ~mask))
    return errs, bad_G, bad_R


BF16_OP_TOL = 3e-3     # BF16 path vs the BF16-operand oracle: per-channel error
BF16_OP_TAU = 5e-3     # ... and its decision band (units of the explore actuators)


def check_bf16_step(gpu, st: O.State, t, nets, p, nets_b, p_b):
    """One BF16-path step from oracle state st compared with the BF16-operand oracle (3e-3,
    outside its 5e-3 band) and with the FP64 oracle (2e-2, outside the fixed 3e-2 band of reading
    R14 and outside the band the BF16 rounding accounts for). Returns (the FP64 oracle's next
    state, worst errors, share of cells in the narrow band)."""
    new, info = O.step(st, nets, t, p)
    new_b, info_b = O.step(st, nets_b, t, p_b)
    mb = band_mask(st, info_b, BF16_OP_TAU, p.rotation)
    errs_b, bG, bR = compare_step(gpu, new_b, mb, BF16_OP_TOL)
    assert bG == 0 and bR == 0 and max(errs_b.values()) <= BF16_OP_TOL, ("vs BF16-operand oracle", errs_b, bG, bR)
    _, bG, bR = compare_step(gpu, new, band_mask(st, info, BF16_TAU, p.rotation), BF16_TOL)
    assert bG == 0 and bR == 0, ("outside the fixed band", bG, bR)
    split, outcome = decision_split(st, info["dir"], info_b["dir"], new.G, new_b.G, new.R, new_b.R)
    m = split | outcome | mb
    errs, bG, bR = compare_step(gpu, new, m, BF16_TOL)
    assert bG == 0 and bR == 0 and max(errs.values()) <= BF16_TOL, ("vs FP64 oracle", errs, bG, bR)
    return new, {"fp64": errs, "bf16_operand": errs_b}, float(m.mean())
