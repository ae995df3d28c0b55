"""Pins of the FP64 oracle against facts fixed outside it: library routines, closed forms,
hand-computed cases, conservation laws and statistics. CPU only."""
import math

import numpy as np
import pytest

from oracle import coral_oracle as O
from oracle import philox as P
from paper_2406_09654_gb300 import worlds


# ----------------------------------------------------------------------------- Philox

@pytest.mark.parametrize("key,ctr", [((1, 2), (0, 0, 0, 0)), ((0xDEADBEEF, 7), (5, 0, 0, 0)),
                                     ((2**64 - 1, 3), (2**64 - 3, 1, 2, 3))])
def test_philox_round_structure_matches_numpy_philox4x64(key, ctr):
    # numpy's Philox is Philox4x64-10 and bumps the counter before each block
    bg = np.random.Philox(key=np.array(key, np.uint64), counter=np.array(ctr, np.uint64))
    raw = bg.random_raw(8)
    c = list(ctr)
    for blk in range(2):
        c[0] = (c[0] + 1) % 2**64
        if c[0] == 0:
            c[1] = (c[1] + 1) % 2**64
        got = P.philox_py(c, key, width=64)
        assert got == [int(v) for v in raw[4 * blk:4 * blk + 4]]


def philox_kat():
    """The published Philox4x32-10 known-answer vectors (tests/golden/philox4x32_10_kat.txt)."""
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "philox4x32_10_kat.txt")
    rows = []
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            v = [int(x, 16) for x in line.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    assert len(rows) == 3
    return rows


@pytest.mark.parametrize("i", range(3))
def test_philox4x32_10_known_answer_vectors(i):
    ctr, key, out = philox_kat()[i]
    assert P.philox_py(ctr, key, width=32) == out
    vec = P.philox4x32(*[np.array([c], np.uint64) for c in ctr], key[0], key[1])
    assert [int(v[0]) for v in vec] == out


def test_philox4x32_vector_equals_scalar():
    cells = np.array([0, 1, 2, 77, 2**32 - 1], np.uint64)
    vec = P.philox4x32(cells, 123, (2 << 24) | 4, 9, 0x01234567, 0x89ABCDEF)
    for i, c in enumerate(cells):
        ref = P.philox_py([int(c), 123, (2 << 24) | 4, 9], [0x01234567, 0x89ABCDEF], width=32)
        assert [int(v[i]) for v in vec] == ref


def test_philox4x32_uniformity_chi2():
    words = P.draw(np.arange(1 << 15), 3, 1, 0, 0, 42)
    for w in words:
        hist = np.bincount((w >> 24).astype(np.int64), minlength=256)
        e = len(w) / 256
        chi2 = float(np.sum((hist - e) ** 2 / e))
        assert 180 < chi2 < 340          # 255 dof, about +-4.5 sigma
    # different streams / steps give different words
    a = P.draw(np.arange(64), 3, 0, 0, 0, 42)[0]
    b = P.draw(np.arange(64), 3, 1, 0, 0, 42)[0]
    c = P.draw(np.arange(64), 4, 0, 0, 0, 42)[0]
    assert (a != b).mean() > 0.9 and (a != c).mean() > 0.9


def test_uniform_open_interval_and_box_muller_moments():
    assert P.uniform01(0) == 0.5 * 2.0 ** -24
    assert P.uniform01(0xFFFFFFFF) == 1.0 - 0.5 * 2.0 ** -24
    w = P.draw(np.arange(200000), 0, 2, 0, 0, 5)
    z0, z1 = P.box_muller(P.uniform01(w[0]), P.uniform01(w[1]))
    z = np.concatenate([z0, z1])
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1) < 0.01
    assert abs(np.mean(z ** 4) - 3) < 0.05
    assert abs(np.corrcoef(z0, z1)[0, 1]) < 0.01


def test_threshold():
    assert P.threshold(0.0) == 0
    assert P.threshold(1e-4) == math.floor(1e-4 * 2 ** 32)
    assert P.threshold(1.0) == 0xFFFFFFFF


# ----------------------------------------------------------------------------- bucketing

@pytest.mark.parametrize("cap,n,layout", [(8, 400, "random"), (64, 1000, "random"), (5, 1, "random")])
def test_bucket_is_stable_counting_sort(cap, n, layout):
    rng = np.random.default_rng(n)
    G = rng.integers(0, cap // 2 + 1, n)
    count, off, perm = O.bucket(G, cap)
    assert np.array_equal(count, np.bincount(G, minlength=cap))
    assert np.array_equal(perm, np.argsort(G, kind="stable"))
    assert off[0] == 0 and np.array_equal(off[1:], np.cumsum(count)[:-1])


# ----------------------------------------------------------------------------- sensing

# Hand table of kernel offsets (dx, dy) in rank order for each rotation; north = row above.
HAND_KERNEL = {
    0: [(0, 0), (0, -1), (1, -1), (-1, -1), (1, 0), (-1, 0), (1, 1), (-1, 1), (0, 1)],
    1: [(0, 0), (1, 0), (1, 1), (1, -1), (0, 1), (0, -1), (-1, 1), (-1, -1), (-1, 0)],
    2: [(0, 0), (0, 1), (-1, 1), (1, 1), (-1, 0), (1, 0), (-1, -1), (1, -1), (0, -1)],
    3: [(0, 0), (-1, 0), (-1, -1), (-1, 1), (0, -1), (0, 1), (1, -1), (1, 1), (1, 0)],
}


def encoded_state(W, H, R=None):
    ys, xs = np.mgrid[0:H, 0:W]
    base = (100 * ys + xs).astype(np.float64).ravel()
    C = np.stack([base + 10000 * (2 + k) for k in range(4)])
    Rv = np.zeros(W * H, np.int64) if R is None else np.asarray(R, np.int64).ravel()
    return O.State(W, H, base + 10000 * 0, base + 10000 * 1, C, np.zeros(W * H, np.int64), Rv)


@pytest.mark.parametrize("W,H", [(3, 3), (5, 5), (4, 7)])
@pytest.mark.parametrize("R", [0, 1, 2, 3])
def test_sense_matches_hand_table(W, H, R):
    st = encoded_state(W, H, np.full((H, W), R))
    x = O.sense(st, np.arange(W * H), O.Params(rotation=1))
    for j in range(W * H):
        cx, cy = j % W, j // W
        for rank, (dx, dy) in enumerate(HAND_KERNEL[R]):
            nx, ny = (cx + dx) % W, (cy + dy) % H
            for ch in range(6):
                assert x[j, 6 * rank + ch] == 100 * ny + nx + 10000 * ch


def test_sense_rotation_off_uses_north():
    st = encoded_state(5, 5, np.full((5, 5), 3))
    x_off = O.sense(st, np.arange(25), O.Params(rotation=0))
    st0 = encoded_state(5, 5)
    assert np.array_equal(x_off, O.sense(st0, np.arange(25), O.Params(rotation=1)))


def test_sense_rotation_symmetry():
    # rotating the whole grid a quarter turn clockwise and adding 1 to every rotation
    # leaves every cell's input vector unchanged
    rng = np.random.default_rng(3)
    n = 6
    chans = rng.normal(size=(6, n, n))
    R = rng.integers(0, 4, (n, n))
    rot = lambda a: np.rot90(a, k=-1)      # clockwise for row 0 = north
    def mk(ch, Rg):
        return O.State(n, n, ch[0].ravel(), ch[1].ravel(), ch[2:].reshape(4, -1),
                       np.zeros(n * n, np.int64), Rg.ravel().astype(np.int64))
    x0 = O.sense(mk(chans, R), np.arange(n * n), O.Params()).reshape(n, n, 54)
    x1 = O.sense(mk(np.stack([rot(c) for c in chans]), (rot(R) + 1) % 4),
                 np.arange(n * n), O.Params()).reshape(n, n, 54)
    assert np.array_equal(rot(x0), x1)


# ----------------------------------------------------------------------------- network

def test_network_zero_weights_gives_bias():
    nets = O.Nets(0, np.zeros((1, 10, 54)), np.linspace(-2, 2, 10)[None])
    z = O.network(np.random.default_rng(0).normal(size=(7, 54)), np.zeros(7, np.int64), nets, O.Params())
    assert np.array_equal(z, np.broadcast_to(np.linspace(-2, 2, 10)[None], (7, 10)))


def test_network_orientation_single_connection():
    # one nonzero weight W[o=3][i=17]: only output 3 moves, and only with input 17
    W = np.zeros((1, 10, 54)); W[0, 3, 17] = 0.7
    nets = O.Nets(0, W, np.zeros((1, 10)))
    x = np.zeros((2, 54)); x[0, 17] = 1.0; x[1, 3] = 1.0
    z = O.network(x, np.zeros(2, np.int64), nets, O.Params())
    assert z[0, 3] == pytest.approx(0.7, abs=1e-15)
    assert np.count_nonzero(z) == 1


def test_network_two_layer_brute_force():
    rng = np.random.default_rng(1)
    H = 5
    nets = O.Nets(H, rng.normal(size=(2, H, 54)), rng.normal(size=(2, H)),
                  rng.normal(size=(2, 10, H)), rng.normal(size=(2, 10)))
    x = rng.normal(size=(3, 54)); g = np.array([1, 0, 1])
    a = O.network(x, g, nets, O.Params(hidden=H))
    for c in range(3):
        h = [math.tanh(sum(nets.W1[g[c], k, i] * x[c, i] for i in range(54)) + nets.b1[g[c], k])
             for k in range(H)]
        for o in range(10):
            ref = sum(nets.W2[g[c], o, k] * h[k] for k in range(H)) + nets.b2[g[c], o]
            assert a[c, o] == pytest.approx(ref, rel=1e-13, abs=1e-14)


def test_round_bf16_matches_torch():
    torch = pytest.importorskip("torch")
    v = np.random.default_rng(2).normal(size=10000) * 10.0 ** np.random.default_rng(3).integers(-5, 5, 10000)
    v = np.concatenate([v, [1 + 2 ** -8, 1 + 3 * 2 ** -8, -1 - 2 ** -8, 0.0]])
    ref = torch.tensor(v.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(O.round_bf16(v), ref)
    assert O.round_bf16(1 + 2 ** -8) == 1.0 and O.round_bf16(1 + 3 * 2 ** -8) == 1 + 2 ** -6


# ----------------------------------------------------------------------------- actuator epilogue

def sig(z):
    return 1.0 / (1.0 + math.exp(-z))


def test_com_hand_values():
    a = np.zeros((3, 10))
    a[0, :4] = [3, 4, 0, 0]; a[2, :4] = [0.3, -0.4, 0, 0]
    c = O.com_activation(a)
    assert np.allclose(c[0], [sig(0.6), sig(0.8), 0.5, 0.5], atol=1e-15)
    assert np.allclose(c[1], 0.5, atol=0)
    assert np.allclose(c[2], [sig(0.3), sig(-0.4), 0.5, 0.5], atol=1e-15)


def test_invest_liquidate_hand_values():
    a = np.zeros((3, 10)); a[0, 4] = 0.5; a[0, 5] = 0.2; a[1, 4] = -0.5; a[1, 5] = -1
    a[2, 4] = 1.0; a[2, 5] = 1.0
    E = np.array([1.0, 1.0, 0.3]); I = np.array([0.5, 0.5, 0.9])
    E1, I1 = O.invest_liquidate(E, I, a, O.Params())
    assert E1[0] == pytest.approx(0.96, abs=1e-15) and I1[0] == pytest.approx(0.54, abs=1e-15)
    assert E1[1] == 1.0 and I1[1] == 0.5
    assert E1[2] == pytest.approx(0.3 - 0.03 + 0.09) and I1[2] == pytest.approx(0.9 + 0.03 - 0.09)
    assert np.allclose(E1 + I1, E + I, rtol=0, atol=1e-15)


# ----------------------------------------------------------------------------- hand-built steps

def const_nets(biases):
    """Direct nets with zero weights: genome g's actuators are exactly tanh(biases[g])."""
    b = np.asarray(biases, np.float64)
    return O.Nets(0, np.zeros((len(b), 10, 54)), b)


QUIET = [0, 0, 0, 0, -1, -1, -1, -1, -1, -1]       # no invest, no liquidate, no explore


def explorer(k, strength=1.0):
    b = list(QUIET)
    b[6 + k] = strength
    return b


def flat_state(W, H, E=1.0, I=0.2, G=None, R=None):
    n = W * H
    return O.State(W, H, np.full(n, E), np.full(n, I), np.full((4, n), 0.5),
                   np.zeros(n, np.int64) if G is None else np.asarray(G, np.int64).ravel(),
                   np.zeros(n, np.int64) if R is None else np.asarray(R, np.int64).ravel())


NOFLOW = dict(k_flow=0.0, e_day=0.0, e_night=0.0)


def idx(W, x, y):
    return y * W + x


def test_single_explorer_takes_over_north():
    W = H = 5
    G = np.zeros((H, W), np.int64); G[2, 2] = 1
    I = np.full(W * H, 0.2); I[idx(W, 2, 2)] = 1.0
    st = flat_state(W, H, G=G); st.I = I
    nets = const_nets([QUIET, explorer(0)])
    new, info = O.step(st, nets, 0, O.Params(**NOFLOW))
    x = 0.5 * math.tanh(1.0) * 1.0
    assert new.I[idx(W, 2, 2)] == pytest.approx(1.0 - x, abs=1e-15)
    assert new.I[idx(W, 2, 1)] == pytest.approx(0.2 + x, abs=1e-15)
    assert new.G[idx(W, 2, 1)] == 1 and new.R[idx(W, 2, 1)] == 0
    assert info["n_takeover"] == 1 and info["n_explore"] == 1
    assert new.I.sum() == pytest.approx(st.I.sum(), abs=1e-14)


def test_explorer_too_weak_only_gives_infrastructure():
    W = H = 5
    G = np.zeros((H, W), np.int64); G[2, 2] = 1
    I = np.full(W * H, 0.9); I[idx(W, 2, 2)] = 1.0
    st = flat_state(W, H, G=G); st.I = I
    new, info = O.step(st, const_nets([QUIET, explorer(0)]), 0, O.Params(**NOFLOW))
    x = 0.5 * math.tanh(1.0)
    assert new.G[idx(W, 2, 1)] == 0                              # 0.38 < 0.9: no takeover
    assert new.I[idx(W, 2, 1)] == pytest.approx(0.9 + x, abs=1e-15)
    assert info["n_takeover"] == 0


@pytest.mark.parametrize("R,k,target", [(1, 0, (3, 2)), (1, 1, (2, 3)), (1, 2, (2, 1)),
                                        (1, 3, (1, 2)), (2, 0, (2, 3)), (3, 1, (2, 1)),
                                        (0, 3, (2, 3))])
def test_explore_direction_follows_rotation(R, k, target):
    W = H = 5
    G = np.zeros((H, W), np.int64); G[2, 2] = 1
    Rg = np.zeros((H, W), np.int64); Rg[2, 2] = R
    I = np.full(W * H, 0.05); I[idx(W, 2, 2)] = 1.0
    st = flat_state(W, H, G=G, R=Rg); st.I = I
    new, _ = O.step(st, const_nets([QUIET, explorer(k)]), 0, O.Params(**NOFLOW))
    tj = idx(W, *target)
    assert new.G[tj] == 1
    # rotation of the exploration: absolute direction from explorer to target
    d = {(0, -1): 0, (1, 0): 1, (0, 1): 2, (-1, 0): 3}[(target[0] - 2, target[1] - 2)]
    assert new.R[tj] == d


def test_two_explorers_max_wins_and_exact_tie_goes_north_first():
    W = H = 5
    # target (2,2); explorer A north at (2,1) explores S, explorer B east at (3,2) explores W
    G = np.zeros((H, W), np.int64); G[1, 2] = 1; G[2, 3] = 2
    I = np.full(W * H, 0.01)
    I[idx(W, 2, 1)] = 1.0; I[idx(W, 3, 2)] = 0.8
    st = flat_state(W, H, G=G); st.I = I
    nets = const_nets([QUIET, explorer(3), explorer(3)])   # back from R=0 = south
    # B at R=0 exploring "back" goes south, not west: give B rotation E so back = W
    st.R[idx(W, 3, 2)] = 1
    new, _ = O.step(st, nets, 0, O.Params(**NOFLOW))
    assert new.G[idx(W, 2, 2)] == 1                              # larger x (north) wins
    # exact tie: equal infrastructure -> equal x -> north (first in N,E,S,W) wins
    st2 = st.copy(); st2.I[idx(W, 3, 2)] = 1.0
    new2, info2 = O.step(st2, nets, 0, O.Params(**NOFLOW))
    assert new2.G[idx(W, 2, 2)] == 1
    # both amounts are absorbed by the target
    x = 0.5 * math.tanh(1.0)
    assert new2.I[idx(W, 2, 2)] == pytest.approx(0.01 + 2 * x, abs=1e-15)
    # make east strictly larger: east wins
    st3 = st.copy(); st3.I[idx(W, 3, 2)] = 1.0 + 1e-3
    new3, _ = O.step(st3, nets, 0, O.Params(**NOFLOW))
    assert new3.G[idx(W, 2, 2)] == 2 and new3.R[idx(W, 2, 2)] == 3


def test_explorer_taken_over_while_exploring():
    W = H = 5
    # A at (2,2) explores north into (2,1) (weak); B at (2,3) explores north into A (strong)
    G = np.zeros((H, W), np.int64); G[2, 2] = 1; G[3, 2] = 2
    I = np.full(W * H, 0.9)
    I[idx(W, 2, 2)] = 0.1; I[idx(W, 2, 3)] = 1.0
    st = flat_state(W, H, G=G); st.I = I
    new, info = O.step(st, const_nets([QUIET, explorer(0), explorer(0)]), 0, O.Params(**NOFLOW))
    xa, xb = 0.5 * math.tanh(1) * 0.1, 0.5 * math.tanh(1) * 1.0
    assert new.G[idx(W, 2, 2)] == 2                              # xb = 0.38 > I1(A) = 0.1
    assert new.I[idx(W, 2, 2)] == pytest.approx(0.1 - xa + xb, abs=1e-15)
    assert new.G[idx(W, 2, 1)] == 0                              # xa < 0.9
    assert new.I.sum() == pytest.approx(st.I.sum(), abs=1e-13)


def test_no_explore_when_all_logits_negative_or_no_infrastructure():
    W = H = 4
    st = flat_state(W, H, I=0.0)
    new, info = O.step(st, const_nets([explorer(0)]), 0, O.Params(**NOFLOW))
    assert info["n_explore"] == 0
    st = flat_state(W, H)
    new, info = O.step(st, const_nets([QUIET]), 0, O.Params(**NOFLOW))
    assert info["n_explore"] == 0 and np.array_equal(new.I, st.I)


# ----------------------------------------------------------------------------- energy flow

def test_flow_uniform_infrastructure_closed_form():
    W = H = 16
    rng = np.random.default_rng(4)
    st = flat_state(W, H); st.E = rng.uniform(0, 1, W * H)
    p = O.Params(k_flow=0.2, e_day=0.0, e_night=0.0)
    new, _ = O.step(st, const_nets([QUIET]), 0, p)
    E = st.E.reshape(H, W)
    nb = np.roll(E, 1, 0) + np.roll(E, -1, 0) + np.roll(E, 1, 1) + np.roll(E, -1, 1)
    assert np.allclose(new.E.reshape(H, W), 0.8 * E + 0.05 * nb, rtol=0, atol=1e-15)


def test_flow_fourier_mode_decay():
    W = H = 16
    ys, xs = np.mgrid[0:H, 0:W]
    for kx, ky in [(1, 0), (2, 3), (8, 8)]:
        wx, wy = 2 * np.pi * kx / W, 2 * np.pi * ky / H
        mode = np.cos(wx * xs + wy * ys)
        st = flat_state(W, H); st.E = (1.0 + 0.1 * mode).ravel()
        new, _ = O.step(st, const_nets([QUIET]), 0, O.Params(k_flow=0.2, e_day=0, e_night=0))
        lam = 1 - 0.2 * (1 - (np.cos(wx) + np.cos(wy)) / 2)
        assert np.allclose(new.E.reshape(H, W), 1.0 + 0.1 * lam * mode, atol=1e-14)


def test_flow_conserves_energy_with_random_infrastructure():
    W, H = 11, 9
    rng = np.random.default_rng(5)
    st = flat_state(W, H); st.E = rng.uniform(0, 1, W * H); st.I = rng.uniform(0, 0.5, W * H)
    st.I[::7] = 0.0
    st.I[idx(W, 3, 3)] = st.I[idx(W, 3, 5)] = st.I[idx(W, 2, 4)] = st.I[idx(W, 4, 4)] = 0.0  # S=0 at (3,4)
    new, info = O.step(st, const_nets([QUIET]), 0, O.Params(e_day=0, e_night=0))
    assert abs(new.E.sum() - st.E.sum()) <= 1e-12 * st.E.sum()
    assert info["S"][idx(W, 3, 4)] == 0 and new.E[idx(W, 3, 4)] >= st.E[idx(W, 3, 4)]


# ----------------------------------------------------------------------------- day/night, totals

def test_day_night_totals():
    w = worlds.make_world(width=12, height=10, n_genomes=3, hidden=0, seed=3)
    st = O.State.from_world(w)
    nets = O.Nets.from_dense(w.dense, 0)
    p = O.Params.from_world(w)
    N = st.n
    for t in (0, 99, 100, 150, 199, 200):
        new, _ = O.step(st, nets, t, p)
        before = st.E.sum() + st.I.sum()
        if (t % 200) < 100:
            assert new.E.sum() + new.I.sum() == pytest.approx(before + N * p.e_day, rel=1e-13)
        else:
            assert new.E.sum() / (1 - p.e_night) + new.I.sum() == pytest.approx(before, rel=1e-13)


# ----------------------------------------------------------------------------- CPPN

def genes_with(**kw):
    """genes: w[k][i] for k in (sin, gauss, tanh), i in (x1, y1, x2, y2, bias); v[k]."""
    g = np.zeros(18)
    K = {"sin": 0, "gauss": 1, "tanh": 2}
    Iin = {"x1": 0, "y1": 1, "x2": 2, "y2": 3, "b": 4}
    for name, val in kw.items():
        if name.startswith("v_"):
            g[15 + K[name[2:]]] = val
        else:
            k, i = name.split("_")
            g[5 * K[k] + Iin[i]] = val
    return g


def test_cppn_constant_from_bias_weight():
    g = genes_with(tanh_b=0.7, v_tanh=1.3)
    W1, b1, W2, b2 = O.cppn_weights(g, 32)
    c = 1.3 * math.tanh(0.7)
    assert np.allclose(W1, c / math.sqrt(54), atol=1e-15) and np.allclose(b1, c / math.sqrt(54))
    assert np.allclose(W2, c / math.sqrt(32), atol=1e-15) and np.allclose(b2, c / math.sqrt(32))


def test_cppn_source_x_coordinate():
    g = genes_with(sin_x1=math.pi / 2, v_sin=1.0)
    W1, b1, W2, b2 = O.cppn_weights(g, 64)
    s1, s2 = 1 / math.sqrt(54), 1 / math.sqrt(64)
    # W1[h][i] depends on the input index only: sin(pi/2 * (-1 + 2i/53))
    assert W1[5, 0] == pytest.approx(-s1) and W1[40, 53] == pytest.approx(s1)
    assert W1[0, 26] == pytest.approx(s1 * math.sin(math.pi / 2 * (-1 + 52 / 53)))
    assert np.allclose(W1, W1[0][None, :])
    assert np.allclose(b1, 0.0) and np.allclose(b2, 0.0)
    assert W2[3, 0] == pytest.approx(-s2) and np.allclose(W2, W2[0][None, :])


def test_cppn_target_coordinates():
    g = genes_with(sin_x2=math.pi / 2, v_sin=2.0)
    W1, b1, W2, b2 = O.cppn_weights(g, 16)
    s1 = 1 / math.sqrt(54)
    assert W1[0, 7] == pytest.approx(-2 * s1) and W1[15, 3] == pytest.approx(2 * s1)
    assert np.allclose(W1, W1[:, :1]) and np.allclose(b1, W1[:, 0])
    g = genes_with(gauss_y2=1.0, v_gauss=1.0)
    W1, b1, W2, b2 = O.cppn_weights(g, 16)
    assert np.allclose(W1, 1 / math.sqrt(54)) and np.allclose(W2, math.exp(-1) / 4)
    assert np.allclose(b2, math.exp(-1) / 4)
    g = genes_with(tanh_y1=1.0, v_tanh=1.0)                     # inputs at y1=-1, hidden y1=0
    W1, b1, W2, b2 = O.cppn_weights(g, 16)
    assert np.allclose(W1, math.tanh(-1) / math.sqrt(54)) and np.allclose(W2, 0) and np.allclose(b1, 0)


def test_cppn_single_layer_and_layer_coords():
    assert np.allclose(O.layer_coords(1), [0.0])
    assert np.allclose(O.layer_coords(3), [-1, 0, 1])
    g = genes_with(sin_x2=math.pi / 2, v_sin=1.0)
    W, b, _, _ = O.cppn_weights(g, 0)
    assert W.shape == (10, 54) and W[0, 5] == pytest.approx(-1 / math.sqrt(54))
    assert W[9, 5] == pytest.approx(1 / math.sqrt(54))


# ----------------------------------------------------------------------------- radiation

def rad_world(W=32, H=32, n=4, p_mut=0.0, p_merge=0.0, cap=64, seed=0):
    w = worlds.make_world(width=W, height=H, n_genomes=n, hidden=8, net="cppn", seed=seed,
                          capacity=cap, radiation_every=1, p_mut=p_mut, p_merge=p_merge)
    return w, O.State.from_world(w), O.Genomes.from_genes(w.genes, cap), O.Params.from_world(w)


def test_radiation_hit_count_binomial():
    w, st, gen, p = rad_world(64, 64, p_mut=0.01, cap=200000)
    total = 0
    events = 40
    for t in range(events):
        _, _, _, ev = O.radiation(st, gen, t, p)
        total += ev["n_mut"]
    n = events * st.n
    mean, sd = n * 0.01, math.sqrt(n * 0.01 * 0.99)
    assert abs(total - mean) < 4 * sd


def test_radiation_hit_set_matches_scalar_philox():
    w, st, gen, p = rad_world(16, 16, p_mut=0.05, p_merge=0.05, cap=600)
    _, _, _, ev = O.radiation(st, gen, 7, p)
    thr_m, thr_g = math.floor(0.05 * 2**32), math.floor(0.05 * 2**32)
    for j in range(st.n):
        wm = P.philox_py([j, 7, 0, 0], [p.seed & 0xFFFFFFFF, p.seed >> 32])
        assert ev["hit_mut"][j] == (wm[0] < thr_m)


def test_radiation_slots_children_and_skip():
    w, st, gen, p = rad_world(32, 32, p_mut=0.02, p_merge=0.0, cap=40, seed=2)
    new, ngen, slots, ev = O.radiation(st, gen, 3, p)
    free = [s for s in range(40) if s >= 4]                      # 4 live genomes
    assert slots == free[:len(slots)]
    assert ev["n_skipped"] == max(0, ev["n_hits"] - 36)
    dev = []
    for s, j in zip(slots, ev["hit_cells"]):
        assert new.G[j] == s and ngen.parent[s] == st.G[j]
        dev.append(ngen.genes[s] - gen.genes[st.G[j]])
    dev = np.array(dev)
    assert dev.shape[0] >= 10
    assert 0.04 < dev.std() < 0.06 and abs(dev.mean()) < 0.02


def test_radiation_merge_crossover_genes_from_either_parent():
    w, st, gen, p = rad_world(48, 48, n=16, p_mut=0.0, p_merge=0.05, cap=1000, seed=4)
    new, ngen, slots, ev = O.radiation(st, gen, 11, p)
    assert len(slots) > 5
    for s, j in zip(slots, ev["hit_cells"]):
        a = gen.genes[st.G[j]]
        assert ev["merge"][j]
        child = ngen.genes[s]
        from_self = child == a
        # every gene is one parent's gene; genes not from self equal the partner's
        partners = [gen.genes[st.G[O.neighbour(48, 48, [j], dx, dy)[0]]] for dx, dy in O.DIRS]
        assert any(np.all(from_self | (child == b)) for b in partners)
    # merge never happens between equal genomes: every merging cell has a partner
    # neighbour with another genome
    for j in np.nonzero(ev["merge"])[0]:
        nbs = [st.G[O.neighbour(48, 48, [j], dx, dy)[0]] for dx, dy in O.DIRS]
        assert any(g != st.G[j] for g in nbs)


def test_radiation_no_merge_inside_single_genome():
    w, st, gen, p = rad_world(16, 16, n=1, p_merge=0.5, cap=300)
    _, _, slots, ev = O.radiation(st, gen, 0, p)
    assert ev["n_merge"] == 0 and slots == []


# ----------------------------------------------------------------------------- invariants

def test_invariants_over_a_run():
    w = worlds.make_world(width=20, height=18, n_genomes=6, hidden=8, net="cppn", seed=9,
                          capacity=64, radiation_every=5, p_mut=0.01, p_merge=0.01)
    st = O.State.from_world(w)
    gen = O.Genomes.from_genes(w.genes, 64)
    p = O.Params.from_world(w)
    nets = O.nets_from_genomes(gen, p.hidden)

    def check(t, s, info):
        assert np.all(s.E >= 0) and np.all(s.I >= 0)
        assert np.all((s.C > 0) & (s.C < 1))
        assert np.all((s.R >= 0) & (s.R <= 3))
        assert np.all(np.isfinite(s.E)) and np.all(np.isfinite(s.I))
        assert np.all((s.G >= 0) & (s.G < 64))

    st2, nets, gen, info = O.run(st, nets, gen, 0, 30, p, on_step=check)
    assert len(np.unique(st2.G)) >= 2


def test_step_cells_equals_full_step():
    w = worlds.make_world(width=23, height=17, n_genomes=5, hidden=16, net="cppn", seed=1,
                          random_rotation=True)
    st = O.State.from_world(w)
    p = O.Params.from_world(w)
    nets = O.nets_from_genomes(O.Genomes.from_genes(w.genes, 5), 16)
    full, _ = O.step(st, nets, 5, p)
    cells = np.array([0, 1, 22, 23, 100, 390, 23 * 17 - 1])
    o = O.step_cells(st, nets, 5, p, cells)
    # same arithmetic; only the BLAS blocking of the per-genome matmul may differ
    assert np.allclose(o["E"], full.E[cells], rtol=1e-14, atol=0)
    assert np.allclose(o["I"], full.I[cells], rtol=1e-14, atol=0)
    assert np.array_equal(o["G"], full.G[cells]) and np.array_equal(o["R"], full.R[cells])
    assert np.allclose(o["C"], full.C[:, cells], rtol=1e-14, atol=0)


def test_explore_argmax_on_preactivations_breaks_saturated_ties():
    # actuators 7 and 8 both round to 1.0 in float32 but their pre-activations differ: the
    # maximal actuator is the one with the larger pre-activation
    z = np.zeros((1, 10)); z[0, 6:10] = [-1.0, 12.0, 13.0, 0.5]
    a = np.tanh(z)
    assert a.astype(np.float32)[0, 7] == a.astype(np.float32)[0, 8] == 1.0
    d, amt, margin = O.explore_decision(z, a, np.array([1.0]), np.array([0]), O.Params())
    assert d[0] == 3 and margin[0] == pytest.approx(1.0)          # logit k=2 -> left of north
    assert amt[0] == pytest.approx(0.5 * math.tanh(13.0))


# ----------------------------------------------------------------------------- genetic distance

def test_genetic_distance_closed_forms():
    g = np.random.default_rng(0).normal(size=18)
    assert O.genetic_distance(g, g) == 0.0
    h = g.copy(); h[5] += 0.9
    assert O.genetic_distance(g, h) == pytest.approx(0.4 * 0.9 / 18, abs=1e-15)
    k = np.random.default_rng(1).normal(size=18)
    assert O.genetic_distance(g, k) == pytest.approx(O.genetic_distance(k, g), abs=0)
    m = np.random.default_rng(2).normal(size=18)
    assert O.genetic_distance(g, m) <= O.genetic_distance(g, k) + O.genetic_distance(k, m) + 1e-15


def test_lineage_follows_parents():
    parent = np.array([-1, -1, 0, 2, 1, 3])
    assert O.lineage(parent, 5) == [5, 3, 2, 0]
    assert O.lineage(parent, 4) == [4, 1]
