"""The block form of the general kernels (sweep_rtb.cuh), restated with plain
integers and checked against the terms that Algorithm 1 / Eq. ineq3 define,
written from the STATE INDEX definition of include/lcs_bound.h alone.

Phase 1 stages blocks of sigma^d consecutive values (the lowest d digits of
the state index vary inside a block), lists for each block Y of v_k the
advance sets N of k strings whose other strings S all carry one letter z in
Y's top digit group, and forms for each such (Y, N) the sigma^|S| sums over
the block's digits on N, one per choice of its digits on S.  It files each
sum at row e(z, S), column t of the means table.  Phase 2 reads, for state
(H, t), row e(z, S_z) at column t for every letter z.  Checked here, for
every state of small shapes and every candidate: the entry phase 2 reads was
produced by exactly one task, from the right argument, and its terms are the
multiset Algorithm 1 defines.  Also: the term-offset table's start formula
against a running sum, and that no task files two sums at one entry.
"""
import math

import pytest

from test_general_addressing import decode, defined_terms

K_TILE_VALS, K_MAX_G, K_MAX_BLOCK = 8192, 64, 16384


def blocks_per_tile(sd):
    g = 1 if sd >= 2048 else K_TILE_VALS // sd
    return min(g, K_MAX_G)


def top_sets(Y, topw, s, d):
    top, Z = Y // topw, [0] * s
    for j in range(d - 1, -1, -1):
        Z[top % s] |= 1 << j
        top //= s
    return Z


def count(Y, topw, s, d, ss):
    if ss == 0:
        return 1
    return sum(math.comb(bin(m).count("1"), ss) for m in top_sets(Y, topw, s, d))


def task(Y, topw, s, d, h, ss, r):
    """(N, e, tail base) of task r of block Y with ss kept strings, as the kernel forms them."""
    full, S, zsel = (1 << d) - 1, 0, 0
    if ss > 0:
        Z = top_sets(Y, topw, s, d)
        for z in range(s):
            c = math.comb(bin(Z[z]).count("1"), ss)
            if r < c:
                zsel, mask = z, Z[z]
                break
            r -= c
        n, local, left = bin(mask).count("1"), 0, ss
        for i in range(n - 1, -1, -1):
            if left == 0:
                break
            c = math.comb(i, left)
            if c <= r:
                local |= 1 << i
                r -= c
                left -= 1
        members = [b for b in range(d) if (mask >> b) & 1]
        for i, b in enumerate(members):
            if (local >> i) & 1:
                S |= 1 << b
    N = full ^ S
    e = (zsel << d) | S if S else 0
    tN = tS = 0
    y, w = Y, 1
    for i in range((h - 1) * d):
        c = y % s
        y //= s
        j = d - 1 - i % d
        if (N >> j) & 1:
            tN += c * w
        elif i < (h - 2) * d:
            tS += c * w
        w *= s
    return N, e, tN + s ** d * tS


def s_offset(S, d, lowS, s):
    off, w = 0, 1
    for j in range(d - 1, -1, -1):
        if (S >> j) & 1:
            off += (lowS % s) * w
            lowS //= s
        w *= s
    return off


def start_of(N, s, d):
    """The kernel's closed form of the table position of set N."""
    st, p1 = 0, 1
    for b in range(d):
        if (N >> b) & 1:
            st += s ** bin(N >> (b + 1)).count("1") * p1
        p1 *= s + 1
    return st


def offsets_table(s, d):
    """start[N] by the closed form; offs[start[N] + m] by the kernel's digit deposit."""
    start, offs = [], {}
    for N in range(1 << d):
        st = start_of(N, s, d)
        start.append(st)
        for m in range(s ** bin(N).count("1")):
            off, w, mm = 0, 1, m
            for j in range(d - 1, -1, -1):
                if (N >> j) & 1:
                    off += (mm % s) * w
                    mm //= s
                w *= s
            offs[st + m] = off
    return start, offs


LANES = {2: (5, 32), 3: (3, 27), 4: (2, 16), 5: (2, 25)}  # (lane digits A, live lanes L)


def lane_outputs(s, d, N, start, offs):
    """The lane-digit form (the kernel uses it for sigma = 2; restated for sigma <= 5):
    [(offset of the output's S digits, sorted term offsets)],
    as the writer lanes of a warp file them after the shuffle sum over the advanced lane digits."""
    A, L = LANES[s]
    full, hi = (1 << d) - 1, (1 << (d - A)) - 1
    S = full ^ N
    nlo = sum(1 << p for p in range(A) if (N >> (d - 1 - p)) & 1)
    J, Q = s ** bin(N & hi).count("1"), s ** bin(S & hi).count("1")

    def digits(lane):
        return [(lane // s ** p) % s for p in range(A)]

    out = []
    for q in range(Q):
        offSh = offs[start[S & hi] + q]
        for lane in range(L):
            dl = digits(lane)
            if any(dl[p] for p in range(A) if (nlo >> p) & 1):
                continue  # not a writer
            # the lanes summed into this writer: same digits outside nlo
            group = [l2 for l2 in range(L) if all(digits(l2)[p] == dl[p] for p in range(A) if not (nlo >> p) & 1)]
            terms = sorted(offSh + offs[start[N & hi] + n] + l2 for n in range(J) for l2 in group)
            out.append((offSh + lane, terms))
    return out


def phase1(s, d, h, check, lanes=False):
    """{(e, t): (k, sorted term addresses)} as phase 1 files them (every tile);
    lanes: the lane-digit form of the sums instead of the per-output one."""
    sd, n_tail = s ** d, s ** (d * (h - 1))
    topw = n_tail // sd
    G = blocks_per_tile(sd)
    start, offs = offsets_table(s, d)
    full = (1 << d) - 1
    filed = {}
    n_ty = (n_tail + G - 1) // G
    tiles = [(0, ty) for ty in range(n_ty)] if check else [(k, ty) for k in range(1, d + 1) for ty in range(n_ty)]
    for kk, ty in tiles:
        Y0 = ty * G
        nb = min(G, n_tail - Y0)
        for k in (range(1, d + 1) if check else [kk]):
            ss = d - k
            cnt = [0]
            for b in range(nb):
                cnt.append(cnt[-1] + count(Y0 + b, topw, s, d, ss))
            T, O = s ** k, s ** ss
            if not check:  # the listed tiles (rt_tile_list) are exactly those with a task
                most = max(max(bin(m).count("1") for m in top_sets(Y0 + b, topw, s, d)) for b in range(nb))
                assert (k == d or most >= d - k) == (cnt[nb] > 0)
            for i in range(cnt[nb]):
                b = 0
                while cnt[b + 1] <= i:
                    b += 1
                N, e, tb = task(Y0 + b, topw, s, d, h, ss, i - cnt[b])
                assert bin(N).count("1") == k
                if lanes:
                    for offS, terms in lane_outputs(s, d, N, start, offs):
                        key = (e, tb + offS)
                        assert key not in filed, f"entry {key} filed twice"
                        filed[key] = (k, [(Y0 + b) * sd + x for x in terms])
                    continue
                for o in range(O):
                    offS = s_offset(full ^ N, d, o, s)
                    addrs = sorted((Y0 + b) * sd + offS + offs[start[N] + m] for m in range(T))
                    key = (e, tb + offS)
                    assert key not in filed, f"entry {key} filed twice"
                    filed[key] = (k, addrs)
    return filed


# (7, 2, 2) and (6, 2, 2): several blocks to a tile with a partial last tile
SHAPES = [(2, 6, 2), (3, 4, 2), (4, 3, 2), (7, 2, 2), (6, 2, 2), (2, 3, 3), (3, 3, 3), (2, 4, 3), (2, 2, 4),
          (5, 2, 2)]


# the lane-digit form is restated where it applies: sigma <= 5, d >= its lane digits
CASES = [(sh, form) for sh in SHAPES for form in ("outputs", "lanes")
         if form == "outputs" or (sh[0] in LANES and sh[1] >= LANES[sh[0]][0])]


@pytest.mark.parametrize("check", [False, True])
@pytest.mark.parametrize("shape,form", CASES, ids=lambda v: str(v))
def test_every_state_reads_the_defined_sums(shape, form, check):
    s, d, h = shape
    filed = phase1(s, d, h, check, lanes=form == "lanes")
    n_tail = s ** (d * (h - 1))
    full = (1 << d) - 1
    used = set()
    for x in range(s ** (d * h)):
        Hidx, t = divmod(x, n_tail)
        sets = [0] * s
        hh = Hidx
        for j in range(d - 1, -1, -1):
            sets[hh % s] |= 1 << j
            hh //= s
        strings = decode(x, s, d, h)
        for z in range(s):
            if sets[z] == full:
                continue
            key = ((z << d) | sets[z] if sets[z] else 0, t)
            assert key in filed, f"state {x} letter {z}: entry {key} never filed"
            k, addrs = filed[key]
            want, kk = defined_terms(strings, z, s)
            assert k == kk and addrs == want, (x, z)
            used.add(key)
    assert used == set(filed), "phase 1 files entries no state reads"


@pytest.mark.parametrize("s,d", [(2, 2), (2, 7), (3, 5), (5, 3), (10, 2), (2, 12)])
def test_offset_table_start_is_the_running_sum(s, d):
    total = 0
    for N in range(1 << d):
        assert start_of(N, s, d) == total
        total += s ** bin(N).count("1")
    assert total == (s + 1) ** d  # the table's length
    if s ** d <= K_MAX_BLOCK:
        assert s ** d - 1 < 2 ** 16  # every offset in a block fits the table's 16-bit entries


def test_tiles_and_shared_memory_fit():
    """Every block-form shape's tile fits the kernel's shared-memory opt-in (227 KiB)."""
    for s in range(2, 11):
        for d in range(2, 17):
            sd = s ** d
            if sd > K_MAX_BLOCK:
                continue
            G = blocks_per_tile(sd)

            def smem(nstage):
                return nstage * stage_bytes(sd) + 256 * 20 + (K_MAX_G + 2) * 4 + 128 * 8 + 2 * 8 + 16

            nstage = 2 if smem(2) <= 200 * 1024 else 1
            assert smem(nstage) <= 227 * 1024
            assert G <= K_MAX_G and (G == 1 or G * sd <= K_TILE_VALS)
            assert G == 1 or sd < 2048


def stage_bytes(sd):
    return (blocks_per_tile(sd) * sd * 8 + 8 + 15) // 16 * 16


@pytest.mark.parametrize("sd", [36, 49, 64, 81, 100, 125, 243, 729, 2048, 2187, 6561, 10000, 15625, 16384])
def test_bulk_copies_stay_inside_their_stage_and_vector(sd):
    """The staging copy of a tile of nb blocks at element e0 covers the even-aligned
    range around it: it must fit its stage buffer (with the tile starting at the
    shift), be a whole number of 16-byte units, and is used only inside the vector."""
    G = blocks_per_tile(sd)
    for n_tail in (G, 3 * G + 1, 7 * G - 1):
        n = n_tail * sd
        for ty in range((n_tail + G - 1) // G):
            nb = min(G, n_tail - ty * G)
            e0, vals = ty * G * sd, nb * sd
            shift = e0 & 1
            a0, a1 = e0 - shift, (e0 + vals + 1) & ~1
            nbytes = (a1 - a0) * 8
            assert nbytes % 16 == 0 and a0 % 2 == 0
            assert nbytes <= stage_bytes(sd)
            assert (shift + vals) * 8 <= stage_bytes(sd)
            bulk = a1 <= n
            if not bulk:  # only a last, misaligned tile falls back to plain loads
                assert ty == (n_tail + G - 1) // G - 1 and (e0 + vals) % 2 == 1


@pytest.mark.parametrize("s,d,h", [(2, 6, 2), (3, 4, 2), (7, 2, 2), (2, 3, 3)])
def test_terms_per_state_the_bench_reports(s, d, h):
    """bench.py's note on the general configs states the terms of F per state
    that the first phase sums; it must be the count of the terms it files."""
    import os
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    filed = phase1(s, d, h, False)
    terms = sum(len(addrs) for _, addrs in filed.values())
    assert terms / s ** (d * h) == pytest.approx(bench.general_terms_per_state(s, d), rel=1e-12)


@pytest.mark.parametrize("s", [2, 3, 4, 5])
def test_lane_shuffle_reduction(s):
    """rtb_lane_reduce restated lane by lane: for sigma = 2 an xor shuffle per
    advanced lane digit, else a sum of the sigma lanes that differ in that digit
    (source lanes taken mod 32, as the shuffle does).  Every writer lane (live,
    advanced digits 0) must end with the sum over the live lanes that agree
    with it on the kept digits."""
    A, L = LANES[s]
    for nlo in range(1 << A):
        vals = [(lane * 7919 + 13) % 1009 if lane < L else 0 for lane in range(32)]
        acc = list(vals)
        w = 1
        for p in range(A):
            if (nlo >> p) & 1:
                if s == 2:
                    acc = [acc[lane] + acc[lane ^ w] for lane in range(32)]
                else:
                    new = []
                    for lane in range(32):
                        b0 = lane - ((lane // w) % s) * w
                        new.append(sum(acc[(b0 + c * w) & 31] for c in range(s)))
                    acc = new
            w *= s

        def digits(lane):
            return [(lane // s ** p) % s for p in range(A)]

        for lane in range(L):
            dl = digits(lane)
            if any(dl[p] for p in range(A) if (nlo >> p) & 1):
                continue
            want = sum(vals[l2] for l2 in range(L)
                       if all(digits(l2)[p] == dl[p] for p in range(A) if not (nlo >> p) & 1))
            assert acc[lane] == want, (s, nlo, lane)
