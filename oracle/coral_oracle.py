"""Plain FP64 CPU oracle of one Coralai substrate step — TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg may import, call or
run anything under oracle/. The CUDA library never does, and nothing here imports the
library: the two share only the seeded inputs of ``paper_2406_09654_gb300.worlds`` (which the
*callers* pass in; this module does not import it either).

What it computes (Barbieux & Canaan, "Coralai", Section "System Design" and Section
"Experiment", Fig. 1): in discrete synchronous steps every cell of a toroidal substrate
sends a kernel (a rotation-ordered 3x3 Moore neighbourhood) of sensor channels (energy,
infrastructure, four communication channels) to the dense network selected by its
GenomeIndex; the network's actuator outputs (4 communication, invest, liquidate, 4
directional explore) are turned by the physics into the next substrate: communication is
normalised and passed through a sigmoid, invest/liquidate move mass between energy and
infrastructure, exploration moves infrastructure to the neighbour picked by the maximal
explore actuator and takes it over when it exceeds that cell's infrastructure, energy flows
along infrastructure and follows a day/night cycle; every M steps radiation mutates or
merges CPPN genomes (HyperNEAT, Section "System Design") and the CPPNs regenerate the
dense nets.

The paper gives no equations or constants. Every place where it is silent is settled by a
numbered reading [R1]..[R16]; each function names the readings it follows. The readings:

[R2]  randomness: Philox4x32-10, key = seed, counter = (cell, step, stream<<24|sub, world);
      hit iff word < floor(p 2^32); normals by Box-Muller.
[R3]  kernel order: centre, then offsets by increasing angle from the rotation's forward
      direction (R in {0=N,1=E,2=S,3=W}, north = row above), ties clockwise first.
[R4]  communication: C' = sigmoid(a_k / max(1, ||a_0..3||_2)).
[R5]  invest i = k_inv max(a4,0), liquidate l = k_liq max(a5,0);
      E1 = E - iE + lI, I1 = I + iE - lI.
[R6]  exploration: k* = the maximal explore actuator (first on ties), m = its value; explore
      iff m > 0 and I1 > 0 with x = k_exp m I1 toward d = (R + [0,1,3,2][k*]) mod 4. The
      actuator is picked and m > 0 tested on the pre-activations z6..z9 (tanh is strictly
      increasing, so it is the same actuator and the same sign; comparing z avoids ties made
      by rounding saturated tanh outputs to 1). The explorer loses x,
      the target absorbs every incoming x; the largest incoming x wins (ties N,E,S,W) and
      takes the target over iff x > I1(target): target adopts the explorer's genome and
      rotation d.
[R7]  energy flow: each cell n sends k_f E1_n to its 4 von Neumann neighbours j in shares
      I_t(j) / S_n, S_n = sum of I_t over n's neighbours (nothing if S_n = 0); then day/night:
      + e_day in the first half of each period T, - e_night E in the second half.
[R8]  CPPN: 5 inputs (x1, y1, x2, y2, 1), hidden sin / gauss / tanh, linear output; layers
      at y = -1, 0, +1, nodes at x = -1 + 2i/(n-1); biases queried at (0, 0, x2, y2);
      scale 1/sqrt(fan_in).
[R9]  tanh on the hidden layer and on all 10 outputs.
[R10] radiation at the end of step t when (t+1) mod M = 0; mutation adds sigma N(0,1) to
      all 18 genes; merge-then-mutate when both hit.
[R11] merge partner = von Neumann neighbour (word & 3); no merge with an equal genome;
      uniform crossover by the bits of a Philox word.
[R12] slots: hits in increasing cell order take the lowest free slots (count 0 after the
      step's physics); excess hits are skipped and counted.
[R13] no death rule.
[R14] decisions on floats (the maximal explore actuator, its sign, the winning explorer, the
      takeover compare) are taken on the FP64 values; ``margins`` report how close each
      decision was, so that tests can set aside the near-ties a lower-precision path may
      decide the other way.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np

from . import philox

N_IN = 54
N_OUT = 10
N_GENES = 18

# absolute von Neumann directions, (dx, dy); north is the row above (-y)
DIRS = ((0, -1), (1, 0), (0, 1), (-1, 0))            # N, E, S, W
# the 8 Moore offsets by octant, clockwise from north
OCTANTS = ((0, -1), (1, -1), (1, 0), (1, 1), (0, 1), (-1, 1), (-1, 0), (-1, -1))
# [R3] octant of kernel rank p (1..8) relative to the forward octant: 0, +45, -45, +90, ...
RANK_DELTA = (0, 1, -1, 2, -2, 3, -3, 4)
# [R6] explore logit k -> quarter turns clockwise from forward (fwd, right, left, back),
# i.e. the von Neumann offsets in kernel rank order
EXPLORE_TURN = (0, 1, 3, 2)


@dataclass
class Params:
    hidden: int = 0
    k_inv: float = 0.1
    k_liq: float = 0.1
    k_exp: float = 0.5
    k_flow: float = 0.2
    e_day: float = 0.005
    e_night: float = 0.005
    day_period: int = 200
    rotation: int = 1
    radiation_every: int = 0
    p_mut: float = 0.0
    p_merge: float = 0.0
    sigma_mut: float = 0.05
    seed: int = 0
    world: int = 0
    # "fp64": exact network; "bf16": network operands (x, W1 with b1, h, W2) rounded to
    # bfloat16, products summed exactly, b2 kept exact — the arithmetic a BF16 tensor-core
    # network with an FP32 bias epilogue defines.
    net_precision: str = "fp64"

    @classmethod
    def from_world(cls, w, **kw):
        ph = dict(w.physics)
        p = cls(hidden=w.hidden, seed=w.seed)
        for k, v in ph.items():
            if hasattr(p, k):
                setattr(p, k, type(getattr(p, k))(v))
        return replace(p, **kw)


@dataclass
class State:
    width: int
    height: int
    E: np.ndarray        # [N] float64
    I: np.ndarray        # [N] float64
    C: np.ndarray        # [4][N] float64
    G: np.ndarray        # [N] int64
    R: np.ndarray        # [N] int64

    @classmethod
    def from_world(cls, w):
        return cls(w.width, w.height, w.E.astype(np.float64).ravel(),
                   w.I.astype(np.float64).ravel(),
                   w.C.astype(np.float64).reshape(4, -1),
                   w.G.astype(np.int64).ravel(), w.R.astype(np.int64).ravel())

    def copy(self):
        return State(self.width, self.height, self.E.copy(), self.I.copy(), self.C.copy(),
                     self.G.copy(), self.R.copy())

    @property
    def n(self):
        return self.width * self.height


@dataclass
class Nets:
    """Dense nets per genome slot. hidden = 0: W1 is [cap][10][54], b1 [cap][10], no layer 2."""
    hidden: int
    W1: np.ndarray
    b1: np.ndarray
    W2: np.ndarray | None = None
    b2: np.ndarray | None = None

    @classmethod
    def from_dense(cls, dense, hidden, capacity=None):
        dense = np.asarray(dense, np.float64)
        n = dense.shape[0]
        cap = capacity or n
        H = hidden
        if H == 0:
            W1 = np.zeros((cap, N_OUT, N_IN)); b1 = np.zeros((cap, N_OUT))
            W1[:n] = dense[:, :N_OUT * N_IN].reshape(n, N_OUT, N_IN)
            b1[:n] = dense[:, N_OUT * N_IN:]
            return cls(0, W1, b1)
        W1 = np.zeros((cap, H, N_IN)); b1 = np.zeros((cap, H))
        W2 = np.zeros((cap, N_OUT, H)); b2 = np.zeros((cap, N_OUT))
        o = 0
        W1[:n] = dense[:, o:o + H * N_IN].reshape(n, H, N_IN); o += H * N_IN
        b1[:n] = dense[:, o:o + H]; o += H
        W2[:n] = dense[:, o:o + N_OUT * H].reshape(n, N_OUT, H); o += N_OUT * H
        b2[:n] = dense[:, o:o + N_OUT]
        return cls(H, W1, b1, W2, b2)


@dataclass
class Genomes:
    """CPPN genome table: genes [cap][18], parent slot [cap] (-1 = loaded, not born)."""
    genes: np.ndarray
    parent: np.ndarray = field(default=None)

    @classmethod
    def from_genes(cls, genes, capacity):
        g = np.zeros((capacity, N_GENES))
        g[:len(genes)] = np.asarray(genes, np.float64)
        return cls(g, np.full(capacity, -1, np.int64))

    def copy(self):
        return Genomes(self.genes.copy(), self.parent.copy())


# --------------------------------------------------------------------------------------
# torus addressing
# --------------------------------------------------------------------------------------

def neighbour(width, height, cells, dx, dy):
    """Flat index of the cell at offset (dx, dy) from each cell, with wrap-around."""
    cells = np.asarray(cells, np.int64)
    x = cells % width
    y = cells // width
    return ((y + dy) % height) * width + (x + dx) % width


def kernel_octant(R, rank, rotation):
    """[R3] octant (0..7, clockwise from north) of kernel rank 1..8 for rotation R."""
    fwd = 2 * (np.asarray(R, np.int64) if rotation else np.zeros_like(R, dtype=np.int64))
    return (fwd + RANK_DELTA[rank - 1]) % 8


# --------------------------------------------------------------------------------------
# a1  sensing (Section "System Design": Kernel of Sensor channels; Section "Experiment")
# --------------------------------------------------------------------------------------

def sense(st: State, cells, p: Params):
    """x[c, 6*rank + ch]: the 6 sensor channels (E, I, C0..C3) at the 9 kernel offsets of each
    cell, centre first and then by increasing angular distance to the cell's rotation [R3]."""
    cells = np.asarray(cells, np.int64)
    chans = [st.E, st.I, st.C[0], st.C[1], st.C[2], st.C[3]]
    x = np.empty((len(cells), N_IN))
    for ch in range(6):
        x[:, ch] = chans[ch][cells]
    for rank in range(1, 9):
        octs = kernel_octant(st.R[cells], rank, p.rotation)
        src = np.empty(len(cells), np.int64)
        for o in range(8):
            sel = octs == o
            if sel.any():
                dx, dy = OCTANTS[o]
                src[sel] = neighbour(st.width, st.height, cells[sel], dx, dy)
        for ch in range(6):
            x[:, 6 * rank + ch] = chans[ch][src]
    return x


# --------------------------------------------------------------------------------------
# a2  network (Section "System Design": GenomeIndex locates the net; HyperNEAT nets)
# --------------------------------------------------------------------------------------

def round_bf16(a):
    """Round to the nearest bfloat16 (ties to even), via the float32 value; returned as FP64."""
    f = np.asarray(a, np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + np.uint64(0x7FFF) + ((u >> np.uint64(16)) & np.uint64(1))) & np.uint64(0xFFFF0000)
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def network(x, genome, nets: Nets, p: Params):
    """Output pre-activations z = W x + b (hidden = 0) or z = W2 tanh(W1 x + b1) + b2, with
    the weights of each cell's genome slot; the actuators are a = tanh(z) [R9]."""
    a = np.empty((len(x), N_OUT))
    bf = p.net_precision == "bf16"
    xin = round_bf16(x) if bf else x
    for g in np.unique(genome):
        rows = genome == g
        W1, b1 = nets.W1[g], nets.b1[g]
        if bf:
            W1, b1 = round_bf16(W1), round_bf16(b1)
        z = xin[rows] @ W1.T + b1
        if nets.hidden == 0:
            a[rows] = z
            continue
        h = np.tanh(z)
        W2 = nets.W2[g]
        if bf:
            h, W2 = round_bf16(h), round_bf16(W2)
        a[rows] = h @ W2.T + nets.b2[g]
    return a


# --------------------------------------------------------------------------------------
# a3..a5  actuator epilogue (Section "Experiment")
# --------------------------------------------------------------------------------------

def com_activation(a):
    """[R4] communication: normalise the 4 com actuators by max(1, L2 norm), then sigmoid."""
    com = a[:, 0:4]
    norm = np.maximum(1.0, np.sqrt(np.sum(com * com, axis=1)))
    return 1.0 / (1.0 + np.exp(-(com / norm[:, None])))


def invest_liquidate(E, I, a, p: Params):
    """[R5] invest moves i*E from energy to infrastructure, liquidate moves l*I back."""
    inv = p.k_inv * np.maximum(a[:, 4], 0.0)
    liq = p.k_liq * np.maximum(a[:, 5], 0.0)
    E1 = E - inv * E + liq * I
    I1 = I + inv * E - liq * I
    return E1, I1


def explore_decision(z, a, I1, R, p: Params):
    """[R6] pick the maximal explore actuator; explore iff it is positive and I1 > 0.
    z, a: pre-activations and actuators. Returns (direction 0..3 or -1, amount, margin). The
    decision compares the FP64 values [R14]; the margin is the smaller of (top1 - top2) and
    |top1| of the pre-activations."""
    logits = z[:, 6:10]
    k = np.argmax(logits, axis=1)                    # first maximum
    zm = logits[np.arange(len(z)), k]
    m = a[np.arange(len(a)), 6 + k]
    go = (zm > 0) & (I1 > 0)
    turn = np.asarray(EXPLORE_TURN)[k]
    Rv = R if p.rotation else np.zeros_like(R)
    d = np.where(go, (Rv + turn) % 4, -1)
    amt = np.where(go, p.k_exp * m * I1, 0.0)
    srt = np.sort(logits, axis=1)
    margin = np.minimum(srt[:, 3] - srt[:, 2], np.abs(srt[:, 3]))
    margin = np.where(I1 > 0, margin, np.inf)
    return d.astype(np.int64), amt, margin


# --------------------------------------------------------------------------------------
# pass 1 / pass 2 of one synchronous step
# --------------------------------------------------------------------------------------

def flow_denominator(st: State, cells):
    """[R7] S_n = sum of I_t over the 4 von Neumann neighbours of n."""
    S = np.zeros(len(cells))
    for dx, dy in DIRS:
        S = S + st.I[neighbour(st.width, st.height, cells, dx, dy)]
    return S


def pass1(st: State, nets: Nets, cells, p: Params):
    """Stages a1..a6 for the given cells; results in full-length arrays (NaN elsewhere)."""
    n = st.n
    cells = np.asarray(cells, np.int64)
    x = sense(st, cells, p)
    z = network(x, st.G[cells], nets, p)
    a = np.tanh(z)
    out = {k: np.full(n, np.nan) for k in ("E1", "I1", "amt", "S", "margin")}
    out["dir"] = np.full(n, -2, np.int64)
    out["C"] = np.full((4, n), np.nan)
    out["a"] = np.full((n, N_OUT), np.nan)
    out["z"] = np.full((n, N_OUT), np.nan)
    E1, I1 = invest_liquidate(st.E[cells], st.I[cells], a, p)
    d, amt, margin = explore_decision(z, a, I1, st.R[cells], p)
    out["E1"][cells], out["I1"][cells] = E1, I1
    out["dir"][cells], out["amt"][cells], out["margin"][cells] = d, amt, margin
    out["S"][cells] = flow_denominator(st, cells)
    out["C"][:, cells] = com_activation(a).T
    out["a"][cells] = a
    out["z"][cells] = z
    return out


def day_night(E2, t, p: Params):
    """[R7] square-wave day/night: + e_day during the first half of each period, then
    - e_night * E during the second half."""
    if (t % p.day_period) * 2 < p.day_period:
        return E2 + p.e_day
    return E2 - p.e_night * E2


def pass2(st: State, p1, cells, t, p: Params):
    """Stages a7..a9 for the given cells from pass-1 values of them and their neighbours."""
    W, H = st.width, st.height
    cells = np.asarray(cells, np.int64)
    m = len(cells)
    I1 = p1["I1"][cells]
    # a7 exploration: incoming explorers, winner, takeover [R6]
    I2 = I1 - p1["amt"][cells]
    best_x = np.full(m, -np.inf)
    best_n = np.full(m, -1, np.int64)
    xs = np.full((4, m), -np.inf)            # incoming amount per direction (-inf: none)
    Is = np.zeros((4, m))                    # I1 of the explorer it comes from
    for D, (dx, dy) in enumerate(DIRS):
        nb = neighbour(W, H, cells, dx, dy)
        inc = p1["dir"][nb] == (D + 2) % 4          # neighbour north of me exploring south...
        xin = np.where(inc, p1["amt"][nb], 0.0)
        I2 = I2 + xin
        xs[D] = np.where(inc, xin, -np.inf)
        Is[D] = np.where(inc, p1["I1"][nb], 0.0)
        win = inc & (xin > best_x)                   # strict: earlier direction keeps ties
        best_x = np.where(win, xin, best_x)
        best_n = np.where(win, nb, best_n)
    take = (best_n >= 0) & (best_x > I1)
    G2 = st.G[cells].copy()
    R2 = st.R[cells].copy()
    G2[take] = st.G[best_n[take]]
    R2[take] = p1["dir"][best_n[take]]
    # margins of the winner and takeover compares: relative to the compared amounts, and in
    # units of the explore actuators (an amount x = k_exp m I1 moves by at most k_exp I1 per
    # unit change of m); the smaller of the two
    has = best_n >= 0
    order = np.argsort(-xs, axis=0, kind="stable")
    col = np.arange(m)
    x1, x2 = xs[order[0], col], xs[order[1], col]
    i1, i2 = Is[order[0], col], Is[order[1], col]
    bx = np.where(has, x1, 0.0)
    rel = np.maximum(np.maximum(np.abs(bx), np.abs(I1)), 1e-30)
    tmargin = np.where(has, np.abs(bx - I1) / np.maximum(rel, p.k_exp * i1), np.inf)
    two = np.isfinite(x2)
    d12 = np.where(two, x1 - np.where(two, x2, 0.0), np.inf)
    rel2 = np.maximum(np.abs(bx), 1e-30)
    z2 = np.maximum(p.k_exp * (i1 + i2), 1e-30)
    tmargin = np.minimum(tmargin, np.where(two, d12 / np.maximum(rel2, z2), np.inf))
    # a8 energy flow along infrastructure [R7]
    E1 = p1["E1"][cells]
    S = p1["S"][cells]
    E2 = E1 - np.where(S > 0, p.k_flow * E1, 0.0)
    for dx, dy in DIRS:
        nb = neighbour(W, H, cells, dx, dy)
        Sn = p1["S"][nb]
        share = np.where(Sn > 0, st.I[cells] / np.where(Sn > 0, Sn, 1.0), 0.0)
        E2 = E2 + p.k_flow * p1["E1"][nb] * share
    # a9 day/night [R7]
    E3 = day_night(E2, t, p)
    return dict(E=E3, I=I2, C=p1["C"][:, cells], G=G2, R=R2, take=take,
                explore=p1["dir"][cells] >= 0, tmargin=tmargin)


def step(st: State, nets: Nets, t: int, p: Params):
    """One full synchronous step t (no radiation). Returns (new state, info)."""
    cells = np.arange(st.n, dtype=np.int64)
    p1 = pass1(st, nets, cells, p)
    o = pass2(st, p1, cells, t, p)
    new = State(st.width, st.height, o["E"], o["I"], o["C"], o["G"], o["R"])
    info = dict(stats=totals(new), n_explore=int(o["explore"].sum()),
                n_takeover=int(o["take"].sum()), margin_explore=p1["margin"],
                margin_target=o["tmargin"], dir=p1["dir"], amt=p1["amt"], a=p1["a"], z=p1["z"],
                E1=p1["E1"], I1=p1["I1"], S=p1["S"])
    return new, info


def step_cells(st: State, nets: Nets, t: int, p: Params, cells):
    """The step's outputs at the listed cells only (no radiation): pass 1 runs on those cells
    and their von Neumann neighbours, pass 2 on the cells. Same arithmetic as ``step``."""
    cells = np.asarray(cells, np.int64)
    need = [cells] + [neighbour(st.width, st.height, cells, dx, dy) for dx, dy in DIRS]
    p1 = pass1(st, nets, np.unique(np.concatenate(need)), p)
    o = pass2(st, p1, cells, t, p)
    o["margin_explore"] = p1["margin"][cells]
    o["margin_explore_nb"] = np.min(
        [p1["margin"][nb] for nb in need[1:]] + [p1["margin"][cells]], axis=0)
    o["pass1"] = p1
    return o


def totals(st: State):
    """a10 global totals in FP64: sum E, sum I, sum C_k."""
    return dict(E=float(np.sum(st.E)), I=float(np.sum(st.I)),
                C=[float(np.sum(st.C[k])) for k in range(4)])


# --------------------------------------------------------------------------------------
# a0  bucketing: stable counting sort of cells by genome slot
# --------------------------------------------------------------------------------------

def bucket(G, capacity):
    """count[g] = cells of slot g; off = exclusive prefix sum of count; perm lists the cells
    of slot 0 in increasing order, then slot 1, ... (stable counting sort, written out)."""
    G = np.asarray(G, np.int64).ravel()
    count = np.zeros(capacity, np.int64)
    for g in G:
        count[g] += 1
    off = np.zeros(capacity, np.int64)
    run = 0
    for g in range(capacity):
        off[g] = run
        run += count[g]
    nxt = off.copy()
    perm = np.empty(len(G), np.int64)
    for j, g in enumerate(G):
        perm[nxt[g]] = j
        nxt[g] += 1
    return count, off, perm


# --------------------------------------------------------------------------------------
# a12  CPPN -> dense weights (Section "System Design": HyperNEAT)
# --------------------------------------------------------------------------------------

def cppn(genes, x1, y1, x2, y2):
    """[R8] CPPN value at a connection: hidden sin / gauss / tanh of w_k . (x1,y1,x2,y2,1),
    output = sum_k v_k h_k."""
    g = np.asarray(genes, np.float64)
    w = g[:15].reshape(3, 5)
    v = g[15:18]
    z = [w[k, 0] * x1 + w[k, 1] * y1 + w[k, 2] * x2 + w[k, 3] * y2 + w[k, 4] for k in range(3)]
    return v[0] * np.sin(z[0]) + v[1] * np.exp(-z[1] * z[1]) + v[2] * np.tanh(z[2])


def layer_coords(n):
    """[R8] x position of the i-th of n nodes of a layer: -1 + 2i/(n-1); a lone node sits at 0."""
    if n == 1:
        return np.zeros(1)
    return -1.0 + 2.0 * np.arange(n) / (n - 1)


def cppn_weights(genes, hidden):
    """[R8] Query one genome's CPPN at every connection of its dense net.
    Inputs at y=-1, hidden at y=0, outputs at y=+1; biases at (0, 0, x2, y2)."""
    xin = layer_coords(N_IN)
    xo = layer_coords(N_OUT)
    if hidden == 0:
        s = 1.0 / np.sqrt(N_IN)
        W = s * cppn(genes, xin[None, :], -1.0, xo[:, None], 1.0)
        b = s * cppn(genes, 0.0, 0.0, xo, 1.0)
        return W, b, None, None
    xh = layer_coords(hidden)
    s1 = 1.0 / np.sqrt(N_IN)
    s2 = 1.0 / np.sqrt(hidden)
    W1 = s1 * cppn(genes, xin[None, :], -1.0, xh[:, None], 0.0)
    b1 = s1 * cppn(genes, 0.0, 0.0, xh, 0.0)
    W2 = s2 * cppn(genes, xh[None, :], 0.0, xo[:, None], 1.0)
    b2 = s2 * cppn(genes, 0.0, 0.0, xo, 1.0)
    return W1, b1, W2, b2


def nets_from_genomes(gen: Genomes, hidden, slots=None, nets: Nets | None = None):
    """Generate (or regenerate the listed slots of) the dense nets from the CPPN genes."""
    cap = len(gen.genes)
    if nets is None:
        if hidden == 0:
            nets = Nets(0, np.zeros((cap, N_OUT, N_IN)), np.zeros((cap, N_OUT)))
        else:
            nets = Nets(hidden, np.zeros((cap, hidden, N_IN)), np.zeros((cap, hidden)),
                        np.zeros((cap, N_OUT, hidden)), np.zeros((cap, N_OUT)))
    for s in (range(cap) if slots is None else slots):
        W1, b1, W2, b2 = cppn_weights(gen.genes[s], hidden)
        nets.W1[s], nets.b1[s] = W1, b1
        if hidden:
            nets.W2[s], nets.b2[s] = W2, b2
    return nets


# --------------------------------------------------------------------------------------
# a11  radiation: mutation and merge of CPPN genomes (Fig. 1 C; Section "System Design")
# --------------------------------------------------------------------------------------

def mutation_normals(cell, t, p: Params):
    """18 standard normals of one cell's mutation: Philox stream 2, subs 0..4, word pairs
    (u0,u1), (u2,u3), ... through Box-Muller [R2]."""
    words = []
    for sub in range(5):
        words += [int(w[0]) for w in philox.draw([cell], t, philox.STREAM_GAUSS, sub,
                                                 p.world, p.seed)]
    u = philox.uniform01(np.array(words[:N_GENES], np.uint64))
    z = np.empty(N_GENES)
    for i in range(N_GENES // 2):
        z[2 * i], z[2 * i + 1] = philox.box_muller(u[2 * i], u[2 * i + 1])
    return z


def radiation(st: State, gen: Genomes, t: int, p: Params):
    """[R10]-[R12] one radiation event on the post-physics state of step t. Returns the new
    state, the new genome table, the new slots (in hit order) and event counts."""
    n = st.n
    cells = np.arange(n, dtype=np.int64)
    thr_mut = philox.threshold(p.p_mut)
    thr_merge = philox.threshold(p.p_merge)
    wm = philox.draw(cells, t, philox.STREAM_MUTATE, 0, p.world, p.seed)
    hit_mut = wm[0].astype(np.uint64) < np.uint64(thr_mut)
    wg = philox.draw(cells, t, philox.STREAM_MERGE, 0, p.world, p.seed)
    hit_merge = wg[0].astype(np.uint64) < np.uint64(thr_merge)
    pdir = (wg[1] & 3).astype(np.int64)
    bits = wg[2].astype(np.int64)
    partner = np.empty(n, np.int64)
    for D, (dx, dy) in enumerate(DIRS):
        sel = pdir == D
        partner[sel] = neighbour(st.width, st.height, cells[sel], dx, dy)
    gp = st.G[partner]
    merge = hit_merge & (gp != st.G)
    hits = np.nonzero(merge | hit_mut)[0]
    count = np.bincount(st.G, minlength=len(gen.genes))
    free = np.nonzero(count == 0)[0]
    n_assign = min(len(hits), len(free))
    new_st = st.copy()
    new_gen = gen.copy()
    slots = []
    for i in range(n_assign):
        j = int(hits[i])
        parent = int(st.G[j])
        child = gen.genes[parent].copy()
        if merge[j]:
            for k in range(N_GENES):
                if (bits[j] >> k) & 1:
                    child[k] = gen.genes[gp[j]][k]
        if hit_mut[j]:
            child = child + p.sigma_mut * mutation_normals(j, t, p)
        s = int(free[i])
        new_gen.genes[s] = child
        new_gen.parent[s] = parent
        new_st.G[j] = s
        slots.append(s)
    ev = dict(n_mut=int(hit_mut.sum()), n_merge=int(merge.sum()), n_hits=len(hits),
              n_assigned=n_assign, n_skipped=len(hits) - n_assign,
              hit_cells=hits, merge=merge, hit_mut=hit_mut)
    return new_st, new_gen, slots, ev


# --------------------------------------------------------------------------------------
# genetic similarity and phylogeny (Section "Discussion and Future Work": NEAT's measure of
# genetic similarity; phylogeny tracking)
# --------------------------------------------------------------------------------------

NEAT_C3 = 0.4      # weight-difference coefficient of NEAT's compatibility distance


def genetic_distance(ga, gb, c3: float = NEAT_C3):
    """NEAT compatibility distance delta = c1 E/N + c2 D/N + c3 mean|w_a - w_b|; the CPPNs here
    share one topology, so there are no excess (E) or disjoint (D) genes and delta reduces to
    c3 times the mean absolute difference of the matching genes."""
    a = np.asarray(ga, np.float64)
    b = np.asarray(gb, np.float64)
    return c3 * float(np.mean(np.abs(a - b)))


def lineage(parent, slot):
    """Ancestors of a genome slot from the parent column (newest first), ending at a loaded
    genome (parent -1)."""
    out = []
    s = int(slot)
    seen = set()
    while s >= 0 and s not in seen:
        seen.add(s)
        out.append(s)
        s = int(parent[s])
    return out


def run(st: State, nets: Nets, gen: Genomes | None, t0: int, n_steps: int, p: Params,
        on_step=None):
    """n_steps full steps starting at step index t0, radiation and regeneration included."""
    info = None
    for t in range(t0, t0 + n_steps):
        st, info = step(st, nets, t, p)
        if p.radiation_every and (t + 1) % p.radiation_every == 0 and gen is not None:
            st, gen, slots, ev = radiation(st, gen, t, p)
            nets_from_genomes(gen, p.hidden, slots, nets)
            info["radiation"] = ev
        if on_step:
            on_step(t, st, info)
    return st, nets, gen, info
