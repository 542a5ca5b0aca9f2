"""The tile walks of the three symmetric sweeps, restated from their kernels with
plain integer (and float32) arithmetic and checked against brute-force
enumerations.  The GPU parity tests check the kernels' outputs; these check
that the walks visit every live tile exactly once, for every size the
kernels accept.

* sigma = d = 2 (sweep_s2d2.cuh): tile k = (s, A, B) of 16 x 16 (a, beta)
  pairs, thread index = Morton code of (a, beta) low bits, a thread live iff
  a <= beta; the live threads own each orbit representative once, tiles
  below the diagonal (skipped whole) hold none, the eight stored states of
  the orbits partition the stored half, and a warp's 32 tails t = (a, b)
  form one aligned run of 32 tail indices.
* d = 2, sigma = 3, 4, 5 (sweep_d2s.cuh): tile (TA, TB) holds a pair (some
  A <= B) iff TB >= RHO TA, RHO = sigma^(KA - KB); live tile j maps back to
  its row through the root of P(TA) = TA nTB - RHO TA (TA - 1) / 2, estimated
  in float32 and corrected exactly.  Its threads own every pair A <= B once,
  and the pairs' reads and writes, checked against the state index,
  partition v_{t-1} and the output.
* sigma = 2, d = 3 (sweep_d3s.cuh): the sheared box J0 < 2^max(L-3,1),
  J1 < 2^(L-2), J2 < 2^(L-3) with I0 = J0, I1 = J0 + J1, I2 = I1 / 2 +
  ((J2 + 37 row) mod 2^(L-3)) and the live test I1 < 2^(L-2), 4 I0 + 8 I2 <=
  2^L - 1 visits each tile of the 4 x 4 x 8 grid that passes the corner test
  (I0 <= I1, I1 / 2 <= I2, 4 I0 + 8 I2 <= 2^L - 1) exactly once, and every
  orbit representative lies in one of those tiles.  Its 32-bit indices stay
  inside the stored half for every h up to the kernel's limit; its outputs
  partition the stored half, and its reads are the states they stand for.
"""
import pathlib
import re

import numpy as np
import pytest


def _spread2(x):
    """bit i of each entry of x moved to bit 2i (x < 2^16)"""
    y = np.zeros_like(x)
    for i in range(16):
        y |= ((x >> i) & 1) << (2 * i)
    return y


@pytest.mark.parametrize("h", [6, 7, 8, 9, 10, 11])
def test_s2d2_orbit_walk(h):
    L = h - 1
    M = (1 << L) - 1
    tn = (1 << (L - 1)) // 16
    nt = 1 << (2 * L)
    k = np.arange(2 * tn * tn, dtype=np.int64)[:, None]
    tid = np.arange(256, dtype=np.int64)[None, :]
    s, rem = k // (tn * tn), k % (tn * tn)
    A, B = rem // tn, rem % tn
    ia = sum(((tid >> (2 * i + 1)) & 1) << i for i in range(4))
    ib = sum(((tid >> (2 * i)) & 1) << i for i in range(4))
    a, beta = A * 16 + ia, B * 16 + ib
    live = np.broadcast_to(a <= beta, (k.size, 256))
    assert not live[(A > B)[:, 0]].any()  # the skipped tiles hold no representative
    s, a, beta = (np.broadcast_to(x, live.shape)[live] for x in (s, a, beta))
    K = 1 << (h - 2)
    reps = set(zip(s.tolist(), a.tolist(), beta.tolist()))
    assert len(reps) == s.size == K * (K + 1)
    assert reps == {(ss, aa, bb) for ss in (0, 1) for bb in range(K) for aa in range(bb + 1)}
    b = np.where(s == 1, M - beta, beta)
    Ea, Eb = _spread2(a), _spread2(b)
    t, sw = (Ea << 1) | Eb, (Eb << 1) | Ea
    tails = np.stack([t, nt - 1 - t, nt - 1 - sw, sw])  # t, ~t, t', ~t'
    states = [set(np.concatenate([tails[:, j], nt + tails[:, j]]).tolist()) for j in range(t.size)]
    assert sum(len(x) for x in states) == 2 * nt  # orbits are disjoint ...
    assert set().union(*states) == set(range(2 * nt))  # ... and cover the stored half
    # every warp of every tile: its tails t, live or not, are one aligned run of 32
    Ea_all, Eb_all = _spread2(A * 16 + ia), _spread2(np.where(k // (tn * tn) == 1, M - (B * 16 + ib), B * 16 + ib))
    t_all = ((Ea_all << 1) | Eb_all).reshape(k.size, 8, 32)
    assert (np.sort(t_all, axis=2) == (t_all.min(axis=2, keepdims=True) + np.arange(32))).all()
    assert (t_all.min(axis=2) % 32 == 0).all()



@pytest.mark.parametrize("h", [6, 8, 10])
def test_s2d2_reads(h):
    """The sigma = d = 2 sweep's reads (s2d2_orbit, s2d2_sweep_orbit): pair
    yb + c (c = 0, 1) of v_{t-1} is the state (0 x_a, x_b c) of its tail x =
    t, ~t, t', ~t' (the heads-01 state with string 1 advanced); the pairs cover
    the stored half (x < N/2), the diagonal orbits reading theirs twice.
    The quad 4 t + c of v_{t-2} (both strings advanced from heads 00) is read
    once per orbit, inside the stored half.  Counting all 32 threads (in a
    diagonal tile some own no orbit and skip their reads), every stream of a
    warp fills whole aligned runs of 32 values."""
    L = h - 1
    M = (1 << L) - 1
    tn = (1 << (L - 1)) // 16
    nt = 1 << (2 * L)
    k = np.arange(2 * tn * tn, dtype=np.int64)[:, None]
    tid = np.arange(256, dtype=np.int64)[None, :]
    s_, rem = k // (tn * tn), k % (tn * tn)
    A, B = rem // tn, rem % tn
    ia = sum(((tid >> (2 * i + 1)) & 1) << i for i in range(4))
    ib = sum(((tid >> (2 * i)) & 1) << i for i in range(4))
    a = A * 16 + ia
    beta = B * 16 + ib
    b = np.where(s_ == 1, M - beta, beta)
    a, b = np.broadcast_to(a, (k.size, 256)), np.broadcast_to(b, (k.size, 256))
    live = np.broadcast_to(A * 16 + ia <= B * 16 + ib, (k.size, 256))
    Ea, Eb = _spread2(a), _spread2(b)
    maskE = _spread2(np.int64(M))
    Eac, Ebc = maskE - Ea, maskE - Eb
    yb = [(Ea << 1) | (Eb << 2), (Eac << 1) | (Ebc << 2), (Ebc << 1) | (Eac << 2), (Eb << 1) | (Ea << 2)]
    t = (Ea << 1) | Eb

    def index(s0, s1):  # two letter lists, head first
        return sum(s0[p] * 2 ** (2 * (h - 1 - p) + 1) + s1[p] * 2 ** (2 * (h - 1 - p)) for p in range(h))

    def bits(x):
        return [(x >> (L - 1 - p)) & 1 for p in range(L)]

    rng = np.random.default_rng(h)
    rows, cols = np.nonzero(live)
    for q in rng.choice(rows.size, 64, replace=False):
        r, c_ = rows[q], cols[q]
        ta, tb = int(a[r, c_]), int(b[r, c_])
        for y, (x0, x1) in zip(yb, [(ta, tb), (M - ta, M - tb), (M - tb, M - ta), (tb, ta)]):
            for c in (0, 1):
                assert int(y[r, c_]) + c == index([0] + bits(x0), bits(x1) + [c])
        for c in range(4):
            assert 4 * int(t[r, c_]) + c == index(bits(ta) + [c >> 1], bits(tb) + [c & 1])

    reads1 = np.concatenate([y[live] for y in yb])
    reads1 = np.concatenate([reads1, reads1 + 1])
    assert np.array_equal(np.unique(reads1), np.arange(2 * nt))
    quads = t[live]
    assert np.unique(quads).size == quads.size and (4 * quads + 3 < 2 * nt).all()
    # warps: every aligned run of 32 values a stream touches is touched whole
    for stream in [np.stack([y, y + 1], -1) for y in yb] + [4 * t[..., None] + np.arange(4)]:
        w = stream.reshape(k.size, 8, -1)
        for row in w.reshape(-1, w.shape[-1])[:: max(1, w.shape[0] * 8 // 512)]:
            vals = np.unique(row)
            assert vals.size % 32 == 0 and np.array_equal(np.unique(vals // 32).size * 32, vals.size)


D2S_GEO = {3: (3, 2), 4: (2, 2), 5: (2, 1)}  # sigma: (KA, KB)


def d2s_live_tiles_bruteforce(s, L):
    KA, KB = D2S_GEO[s]
    nTA, nTB = s ** (L - KA), s ** (L - KB)
    out = []
    for TA in range(nTA):
        for TB in range(nTB):
            # some A <= B with A in [TA s^KA, +s^KA), B in [TB s^KB, +s^KB)
            if TA * s ** KA <= TB * s ** KB + s ** KB - 1:
                out.append((TA, TB))
    return out


def d2s_live_tile(s, L, j):
    KA, KB = D2S_GEO[s]
    rho, nTB = s ** (KA - KB), s ** (L - KB)

    def P(t):
        return t * nTB - rho * (t * (t - 1) // 2)

    b = np.float32(nTB) + np.float32(0.5) * np.float32(rho)
    disc = max(b * b - np.float32(2.0) * np.float32(rho) * np.float32(j), np.float32(0.0))
    t = max(int((b - np.sqrt(np.float32(disc))) / np.float32(rho)), 0)
    while t > 0 and P(t) > j:
        t -= 1
    while P(t + 1) <= j:
        t += 1
    return t, rho * t + (j - P(t))


@pytest.mark.parametrize("s,L", [(3, 3), (3, 4), (3, 5), (3, 6), (3, 7), (4, 2), (4, 3), (4, 4), (4, 5),
                                 (5, 2), (5, 3), (5, 4)])
def test_d2s_live_tile_walk(s, L):
    want = d2s_live_tiles_bruteforce(s, L)
    KA, KB = D2S_GEO[s]
    nTA, nTB, rho = s ** (L - KA), s ** (L - KB), s ** (KA - KB)
    count = nTA * nTB - rho * (nTA * (nTA - 1) // 2)
    assert count == len(want)
    assert [d2s_live_tile(s, L, j) for j in range(count)] == want  # row order, each once


@pytest.mark.parametrize("s,L", [(3, 11), (4, 9), (5, 7)])
def test_d2s_live_tile_inverse_at_the_largest_sizes(s, L):
    """The float32 estimate plus correction at the largest shapes (sampled)."""
    KA, KB = D2S_GEO[s]
    nTA, nTB, rho = s ** (L - KA), s ** (L - KB), s ** (KA - KB)
    count = nTA * nTB - rho * (nTA * (nTA - 1) // 2)
    rng = np.random.default_rng(L)
    for j in list(range(64)) + list(range(count - 64, count)) + [int(x) for x in rng.integers(0, count, 2000)]:
        TA, TB = d2s_live_tile(s, L, j)
        P = TA * nTB - rho * (TA * (TA - 1) // 2)
        assert 0 <= TA < nTA and rho * TA <= TB < nTB and P <= j < P + (nTB - rho * TA)



def _d2s_pair(s, L, j, r):
    """(A, B) of thread r of live tile j (d2s_pair): the thread index's base-s
    digits are A0, B0, A1, B1, ... with A's surplus digits last."""
    KA, KB = D2S_GEO[s]
    TA, TB = d2s_live_tile(s, L, j)
    ia = ib = 0
    wa = wb = 1
    for i in range(KA + KB):
        dgt = r % s
        r //= s
        if i % 2 == 0 or i // 2 >= KB:
            ia += dgt * wa
            wa *= s
        else:
            ib += dgt * wb
            wb *= s
    return TA * s ** KA + ia, TB * s ** KB + ib


def _spread_s2(x, s, L):
    """base-s digits of x moved to base s^2 positions (d2s_spread)"""
    return sum(((x // s ** i) % s) * s ** (2 * i) for i in range(L))


def _d2_index(s, h, s0, s1):
    """the header's state index of the strings s0, s1 (letter lists, head first)"""
    return sum(s0[p] * s ** (2 * (h - 1 - p) + 1) + s1[p] * s ** (2 * (h - 1 - p)) for p in range(h))


def _letters(x, s, L):
    return [(x // s ** (L - 1 - p)) % s for p in range(L)]


@pytest.mark.parametrize("s,L", [(3, 3), (3, 4), (4, 2), (4, 3), (5, 2), (5, 3)])
def test_d2s_pairs_and_addresses(s, L):
    """The d = 2 swap-aware sweep's pairs and addresses (sweep_d2s.cuh) against
    the state index: every pair A <= B owned once; the reads of P(t, g) and
    P(ts, g) partition v_{t-1} (each value read once), and each is the state
    (g a, b c) of its definition; the block of v_{t-2} is the four-letter
    advance of t; the outputs partition the states; inside a tile the P
    addresses of consecutive threads are s apart (a warp reads one run)."""
    KA, KB = D2S_GEO[s]
    h = L + 1
    nt = s ** (2 * L)
    N = s ** (2 * h)
    nTA, nTB, rho = s ** (L - KA), s ** (L - KB), s ** (KA - KB)
    n_live = nTA * nTB - rho * (nTA * (nTA - 1) // 2)
    T = s ** (KA + KB)
    pairs, reads1, reads2, writes = [], [], [], []
    for j in range(n_live):
        bases = []
        for r in range(T):
            A, B = _d2s_pair(s, L, j, r)
            eA, eB = _spread_s2(A, s, L), _spread_s2(B, s, L)
            bases.append(eA * s + eB * s * s)
            if A > B:
                continue
            pairs.append((A, B))
            t, ts = eA * s + eB, eB * s + eA
            a, b = _letters(A, s, L), _letters(B, s, L)
            sides = [(eA, eB, a, b)] if t == ts else [(eA, eB, a, b), (eB, eA, b, a)]
            for ex, ey, x, y in sides:
                for g in range(s):
                    for c in range(s):
                        addr = g * nt * s + ex * s + ey * s * s + c
                        assert addr == _d2_index(s, h, [g] + x, y + [c])
                        reads1.append(addr)
            for c in range(s * s):
                addr = t * s * s + c
                assert addr == _d2_index(s, h, a + [c // s], b + [c % s])
                reads2.append(addr)
            for H in range(s * s):
                writes.append(H * nt + t)
                if t != ts:
                    writes.append(H * nt + ts)
        assert all(bases[r] - bases[0] == s * r for r in range(T))
    assert sorted(pairs) == [(A, B) for A in range(s ** L) for B in range(A, s ** L)]
    assert sorted(reads1) == list(range(N))
    assert len(set(reads2)) == len(reads2) == len(pairs) * s * s
    assert sorted(writes) == list(range(N))


def d3s_live_tiles_bruteforce(L):
    M = (1 << L) - 1
    out = set()
    for I0 in range(1 << (L - 2)):
        for I1 in range(1 << (L - 2)):
            for I2 in range(1 << (L - 3)):
                if 4 * I0 <= 4 * I1 + 3 and 4 * I1 <= 8 * I2 + 7 and 4 * I0 + 8 * I2 <= M:
                    out.add((I0, I1, I2))
    return out


def d3s_walk(L):
    M = (1 << L) - 1
    n = 1 << (max(L - 3, 1) + 2 * L - 5)
    out = []
    for k in range(n):
        row = k >> (L - 3)
        I0 = k >> (2 * L - 5)
        I1 = I0 + (row & ((1 << (L - 2)) - 1))
        I2 = (I1 >> 1) + ((k + 37 * row) & ((1 << (L - 3)) - 1))
        if I1 < (1 << (L - 2)) and 4 * I0 + 8 * I2 <= M:
            out.append((I0, I1, I2))
    return out


@pytest.mark.parametrize("L", [3, 4, 5, 6, 7, 8])
def test_d3s_sheared_rotated_walk(L):
    walk = d3s_walk(L)
    assert len(walk) == len(set(walk))
    assert set(walk) == d3s_live_tiles_bruteforce(L)


@pytest.mark.parametrize("L", [3, 4, 5, 6])
def test_d3s_every_representative_lies_in_a_live_tile(L):
    """No representative is missed: T0 <= T1 <= T2 and (T0, T1, T2) <= (~T2,
    ~T1, ~T0), i.e. T0 + T2 < 2^L - 1, or T0 + T2 = 2^L - 1 and T1 < 2^(L-1),
    always lies in a live tile (live tiles may also hold none: the kernel's
    per-thread test drops those)."""
    M = (1 << L) - 1
    live = d3s_live_tiles_bruteforce(L)
    n_rep = 0
    for T0 in range(1 << L):
        for T1 in range(T0, 1 << L):
            for T2 in range(T1, 1 << L):
                if T0 + T2 < M or (T0 + T2 == M and T1 < (1 << (L - 1))):
                    n_rep += 1
                    assert (T0 // 4, T1 // 4, T2 // 8) in live
    assert n_rep > 0



def _spread3(x):
    """bit i of x (i < 10, as spread3_32 keeps) moved to bit 3i"""
    assert 0 <= x < 1 << 10
    y = 0
    for i in range(10):
        y |= ((x >> i) & 1) << (3 * i)
    return y


def _tail32(sa, sb, sc):
    return (sa << 2) | (sb << 1) | sc


def _d3s_max_h():
    src = (pathlib.Path(__file__).resolve().parents[1] / "paper_2407_10925_gb300" / "csrc" / "sweep_d3s.cuh").read_text()
    return int(re.search(r"kD3sMaxH\s*=\s*(\d+)", src).group(1))


def test_d3s_sweep_indices_stay_in_the_stored_half():
    """The d = 3 sweep (sweep_d3s.cuh) forms its indices in 32 bits.  Each index
    it reads or writes, up to the last value of a two- or four-value load, lies
    in the stored half (2^(3h-1) = 4 nt states), and that half has at most 2^32
    states for every h up to the kernel's limit.  Spreads and tails are
    monotone in each argument, so the largest index comes from the largest
    components: T0 <= 2^(L-1) - 1 (T0 + T2 <= 2^L - 1 with T0 <= T2), T1 and T2
    up to 2^L - 1, and a complement side's spread at most spread(2^L - 1)."""
    h_max = _d3s_max_h()
    for h in range(4, h_max + 1):
        L = h - 1
        M = (1 << L) - 1
        S_any = _spread3(M)
        S_T0 = _spread3((1 << (L - 1)) - 1)
        nt = 1 << (3 * L)
        top = 1 << (3 * L + 1)
        last = {
            "pair sum, one string advanced": _tail32(S_any, S_any, S_any << 3) + 1,
            "quad sum, two strings advanced": _tail32(S_any, S_any << 3, S_any << 3) + 2 + 1,
            "pair sum at string 1 head 1": (_tail32(S_any, S_any, S_any << 3) | top) + 1,
            "block of eight, both sides": (_tail32(S_T0, S_any, S_any) << 3) + 4 + 2 + 1,
            "output at head 011": 3 * nt + _tail32(S_any, S_any, S_any),
        }
        for name, x in last.items():
            assert x < 4 * nt, (h, name, x)
        assert 4 * nt == 2 ** (3 * h - 1) <= 2 ** 32
        assert top < 2 ** 32 and 1 << (max(L - 3, 1) + 2 * L - 5) < 2 ** 32  # the head bit and the tile count
    assert 2 ** (3 * (h_max + 1) - 1) > 2 ** 32  # the limit is tight



def _d3s_rep(I0, I1, I2, M, L, r):
    """d3s2_rep: the representative of thread pair r of tile (I0, I1, I2), or None"""
    t1 = (r & 1) | (((r >> 3) & 1) << 1)
    t0 = ((r >> 1) & 1) | (((r >> 4) & 1) << 1)
    t2 = ((r >> 2) & 1) | (((r >> 5) & 1) << 1) | (((r >> 6) & 1) << 2)
    T = (4 * I0 + t0, 4 * I1 + t1, 8 * I2 + t2)
    if T[0] > T[1] or T[1] > T[2] or T[0] + T[2] > M:
        return None
    if T[0] + T[2] == M and T[1] >= 1 << (L - 1):
        return None
    return T


PERMS3 = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]


def _dup_mask(e01, e12):
    return 0x3E if e01 and e12 else 0x2C if e01 else 0x32 if e12 else 0


@pytest.mark.parametrize("L", [3, 4, 5, 6])
def test_d3s_outputs_and_reads(L):
    """The sigma = 2, d = 3 sweep (sweep_d3s.cuh), restated: over the walk's
    live tiles and both sides (tau, ~tau) of every orbit pair, the outputs at
    the four stored heads of every distinct permutation partition the stored
    half (string 0's head 0).  On sampled pairs each read is the state it
    stands for, by the header's index: A1[k] the pair (0 X_o, 0 X_o', X_k c)
    of v_{t-1}, A2[k] the quad (0 X_k, X_o c, X_o' c') of v_{t-2}, the block
    the eight (T0 c, T1 c', T2 c'') of v_{t-3}."""
    h = L + 1
    M = (1 << L) - 1
    nt = 1 << (3 * L)

    def tail(sa, sb, sc):
        return (sa << 2) | (sb << 1) | sc

    def index(s0, s1, s2):  # three letter lists, head first
        return sum(s0[p] * 2 ** (3 * (h - 1 - p) + 2) + s1[p] * 2 ** (3 * (h - 1 - p) + 1) + s2[p] * 2 ** (3 * (h - 1 - p))
                   for p in range(h))

    def bits(x):
        return [(x >> (L - 1 - p)) & 1 for p in range(L)]

    writes, reps = [], []
    for k in range(1 << (max(L - 3, 1) + 2 * L - 5)):
        row = k >> (L - 3)
        I0 = k >> (2 * L - 5)
        I1 = I0 + (row & ((1 << (L - 2)) - 1))
        I2 = (I1 >> 1) + ((k + 37 * row) & ((1 << (L - 3)) - 1))
        if not (I1 < (1 << (L - 2)) and 4 * I0 + 8 * I2 <= M):
            continue
        for r in range(128):
            T = _d3s_rep(I0, I1, I2, M, L, r)
            if T is None:
                continue
            reps.append(T)
            dup = _dup_mask(T[0] == T[1], T[1] == T[2])
            for side in (0, 1):
                S = [_spread3(x ^ (M if side else 0)) for x in T]
                for q, (p0, p1, p2) in enumerate(PERMS3):
                    if (dup >> q) & 1:
                        continue
                    x0 = tail(S[p0], S[p1], S[p2])
                    writes.extend(m * nt + x0 for m in range(4))
    assert sorted(writes) == list(range(4 * nt))
    assert len(set(reps)) == len(reps)

    rng = np.random.default_rng(L)
    for i in rng.choice(len(reps), min(40, len(reps)), replace=False):
        T = reps[i]
        for side in (0, 1):
            X = [x ^ (M if side else 0) for x in T]
            S = [_spread3(x) for x in X]
            for kk in range(3):
                o, o2 = (1 if kk == 0 else 0), (1 if kk == 2 else 2)
                for c in (0, 1):
                    assert tail(S[o], S[o2], S[kk] << 3) + c == index([0] + bits(X[o]), [0] + bits(X[o2]), bits(X[kk]) + [c])
                a2 = tail(S[kk], S[o] << 3, S[o2] << 3)
                for c in range(4):
                    assert a2 + c == index([0] + bits(X[kk]), bits(X[o]) + [c >> 1], bits(X[o2]) + [c & 1])
        ST = [_spread3(x) for x in T]
        for side in (0, 1):
            b = (tail(ST[0], ST[1], ST[2]) << 3) + 4 * side
            for c in range(4):
                cc = 4 * side + c
                assert b + c == index(bits(T[0]) + [cc >> 2], bits(T[1]) + [(cc >> 1) & 1], bits(T[2]) + [cc & 1])


def _tri_decode(q):
    """tri_decode (sweep_s2d2.cuh): the upper-triangle index q -> (A, B), A <= B,
    q = B (B + 1) / 2 + A; a double-precision root corrected exactly"""
    b = int((np.sqrt(8.0 * float(q) + 1.0) - 1.0) * 0.5)
    while b * (b + 1) // 2 > q:
        b -= 1
    while (b + 1) * (b + 2) // 2 <= q:
        b += 1
    return q - b * (b + 1) // 2, b


def test_tri_decode_of_the_batch_walk():
    """The batch's sigma = d = 2 items number their upper-triangle tiles with q;
    the decode is exact for every q of the sizes a batch takes and, sampled,
    far beyond them."""
    want = [(A, B) for B in range(700) for A in range(B + 1)]
    assert [_tri_decode(q) for q in range(len(want))] == want
    rng = np.random.default_rng(7)
    for q in [int(v) for v in rng.integers(0, 1 << 52, 3000)] + [(1 << 52) - 1, (1 << 40) + 12345]:
        A, B = _tri_decode(q)
        assert 0 <= A <= B and B * (B + 1) // 2 + A == q
