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


def band_mask(st: O.State, info, tau):
    """Cells whose I, G or R may legitimately differ because a float decision of the oracle
    was within tau of flipping: explorers in band and their 4 possible targets, and target
    cells whose winner or takeover compare was in band."""
    W, H = st.width, st.height
    ex = info["margin_explore"] < tau
    tg = info["margin_target"] < tau
    m = ex.copy() | tg
    idx = np.nonzero(ex)[0]
    for dx, dy in O.DIRS:
        m[O.neighbour(W, H, idx, dx, dy)] = True
    return m


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
