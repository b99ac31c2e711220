"""The split selection's histogram window, checked against the full rule on the CPU.

Reading R3 (Sec. III-A1): over the sorted interval points v_0 <= ... <= v_1023
(the node's strided sample), c_j = #{x < v_j} over the node's points and the
split is v_{j*} with j* = argmin |2 c_j - n|, ties to the smallest j.  The
build's first histogram pass counts bins one by one only for the interval
points of ranks 384..640 and the points below v_384; when 2 c_384 <= n <=
2 c_640 the selection over those counts (zero elsewhere) must give the same
split value and left count as the full histogram, and otherwise the node takes
the full pass.  This test restates both selections in numpy, independently of
the CUDA code and of the oracle, and checks that claim on nodes with heavy
ties, continuous values and samples biased to either side.
"""
import numpy as np

S, LO, HI = 1024, 384, 640


def strided_sample(x):
    n = x.shape[0]
    return np.sort(x[(np.arange(S, dtype=np.int64) * n) // S])


def full_rule(x, v):
    n = x.shape[0]
    xs = np.sort(x)
    c = np.searchsorted(xs, v, side="left")          # c_j = #{x < v_j}
    j = int(np.argmin(np.abs(2 * c.astype(np.int64) - n)))   # first minimum: smallest j
    return v[j], int(c[j])


def window_rule(x, v):
    """Bins as the first pass stores them: bin lo holds #{x < v_lo}; bin b in
    (lo, hi] holds #{x : #{v_i <= x} = b} for v_lo <= x < v_hi; the rest 0.
    Returns None when the crossing lies outside the window."""
    n = x.shape[0]
    h = np.zeros(S + 1, np.int64)
    h[LO] = np.count_nonzero(x < v[LO])
    inw = x[(x >= v[LO]) & (x < v[HI])]
    b = np.searchsorted(v, inw, side="right")        # #{v_i <= x}
    assert b.size == 0 or (b.min() > LO and b.max() <= HI)
    np.add.at(h, b, 1)
    c = np.cumsum(h)[:S]                             # c'_j for j < 1024
    if 2 * c[LO] > n or 2 * c[HI] < n:
        return None
    j = int(np.argmin(np.abs(2 * c - n)))
    return v[j], int(c[j])


def nodes(seed):
    rng = np.random.default_rng(seed)
    for t in range(400):
        n = int(rng.integers(1025, 20000))
        kind = t % 5
        if kind == 0:
            x = rng.random(n, dtype=np.float32)
        elif kind == 1:
            x = rng.integers(0, int(rng.integers(2, 40)), n).astype(np.float32)   # heavy ties
        elif kind == 2:
            x = (rng.standard_normal(n) * 1e-3).astype(np.float32)
        elif kind == 3:
            # strided samples drawn low or high: the crossing leaves the window
            x = rng.random(n, dtype=np.float32)
            pos = (np.arange(S, dtype=np.int64) * n) // S
            x[pos] = x[pos] * np.float32(0.2) + np.float32(0.0 if t % 2 else 0.8)
        else:
            x = np.concatenate([np.full(n // 2, 0.5, np.float32), rng.random(n - n // 2, dtype=np.float32)])
            rng.shuffle(x)
        yield x


def test_window_matches_full_rule():
    agreed = missed = 0
    for x in nodes(7):
        v = strided_sample(x)
        w = window_rule(x, v)
        f = full_rule(x, v)
        if w is None:
            missed += 1
            continue
        agreed += 1
        assert np.float32(w[0]) == np.float32(f[0]) and w[1] == f[1], (w, f)
    # both branches are exercised: the continuous and lightly tied nodes decide in the
    # window; the biased samples and a median tied over half the node take the full pass
    assert agreed >= 200 and missed >= 100


def test_window_rule_catches_a_wrong_window_check():
    """A planted mistake: accepting the window without its check gives a
    different split on some node whose crossing lies outside the window."""
    differs = 0
    for x in nodes(8):
        v = strided_sample(x)
        n = x.shape[0]
        h = np.zeros(S + 1, np.int64)
        h[LO] = np.count_nonzero(x < v[LO])
        np.add.at(h, np.searchsorted(v, x[(x >= v[LO]) & (x < v[HI])], side="right"), 1)
        c = np.cumsum(h)[:S]
        j = int(np.argmin(np.abs(2 * c - n)))
        differs += (v[j], int(c[j])) != full_rule(x, v)
    assert differs > 0


def test_tile_left_counts_from_window_bins():
    """A tile's left count for a split decided in the window is its own count
    below v_384 plus its window bins 385 .. j* (bin b: #{v_i <= x} = b), which
    is how the build counts tiles without reading their column again."""
    checked = 0
    for x in nodes(9):
        v = strided_sample(x)
        if window_rule(x, v) is None:
            continue
        xs = np.sort(x)
        c = np.searchsorted(xs, v, side="left")
        j = int(np.argmin(np.abs(2 * c.astype(np.int64) - x.shape[0])))
        if not (LO <= j <= HI):
            continue
        # cut the node at arbitrary tile boundaries
        cuts = np.sort(np.random.default_rng(j).integers(0, x.shape[0], 5))
        for t in np.split(x, cuts):
            below = np.count_nonzero(t < v[LO])
            b = np.searchsorted(v, t[(t >= v[LO]) & (t < v[HI])], side="right")
            bins = np.bincount(b - LO - 1, minlength=HI - LO)
            assert below + int(bins[: j - LO].sum()) == np.count_nonzero(t < v[j])
            checked += 1
    assert checked > 1000
