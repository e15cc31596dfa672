"""Pins of the oracle's block coder: area order (Eq. 1), area symbols
(Eq. 2), SMR bitplanes, empty-plane removal, zero runs and counter width
(Eq. 3), Huffman code and tree (Fig. 3), against hand-worked fixtures,
invariants and an independent parse of the bytes.
"""
import heapq
import itertools
import os

import numpy as np
import pytest

from blockparse import parse_block

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


# ---------------------------------------------------------------- Eq. 1
def test_eq1_golden_w8_h8(orc):
    for k, i, j, p in _rows("eq1_area_order_w8_h8.txt"):
        assert orc.area_T(int(k), 8, 8) == (int(i), int(j), int(p))


@pytest.mark.parametrize("w,h,d", [(4, 4, 1), (8, 4, 3), (4, 12, 2), (16, 8, 4), (128, 128, 2), (20, 36, 3)])
def test_eq1_is_a_bijection_onto_areas_and_planes(orc, w, h, d):
    n = w * h // 8
    seen = set()
    prev_p = 0
    for k in range(d * n):
        i, j, p = orc.area_T(k, w, h)
        assert 0 <= i <= h - 2 and i % 2 == 0 and 0 <= j <= w - 4 and j % 4 == 0
        # the printed column formula holds as printed
        assert j == 4 * ((k // 2) % (w // 4))
        assert p >= prev_p            # sign plane first, then one plane after another
        prev_p = p
        seen.add((i, j, p))
    assert len(seen) == d * n


# ---------------------------------------------------------------- Eq. 2
def test_eq2_golden_symbols(orc):
    for top, bot, sym in _rows("eq2_area_symbols.txt"):
        area = np.array([[int(c) for c in top], [int(c) for c in bot]], np.int64)
        # one magnitude bit plane, d = 2: value 1 sets plane 1
        assert orc.area_symbol(area, 0, 0, 1, 2) == int(sym), (top, bot)


def test_eq2_is_a_bijection_of_patterns(orc):
    syms = set()
    for bits in itertools.product((0, 1), repeat=8):
        area = np.array(bits, np.int64).reshape(2, 4)
        s = orc.area_symbol(area, 0, 0, 1, 2)
        inv = orc.area_symbol(1 - area, 0, 0, 1, 2)
        assert s + inv == 255
        syms.add(s)
    assert syms == set(range(256))


def test_smr_planes_sign_then_msb_to_lsb(orc):
    # single coefficient -5 (magnitude 101b) at the top-left of a 4x4 block:
    # d = 1 + bitlen(5) = 4; planes: sign, bit 2, bit 1, bit 0
    blk = np.zeros((1, 4, 4), np.int64)
    blk[0, 0, 0] = -5
    data, st = orc.encode_block(blk)
    assert st["d"] == 4
    parsed = parse_block(data, 1, 4, 4)
    syms = [None if parsed["planes"][p] is None else parsed["planes"][p]["symbols"][0] for p in range(4)]
    assert syms == [1, 1, None, 1]     # plane for bit 1 is all zero -> removed
    assert parsed["removed"] == [[0, 0, 1, 0]]


# ------------------------------------------------------------- Huffman
def optimal_cost(freq):
    h = [f for f in freq if f > 0]
    if len(h) <= 1:
        return 0
    heapq.heapify(h)
    cost = 0
    while len(h) > 1:
        a, b = heapq.heappop(h), heapq.heappop(h)
        cost += a + b
        heapq.heappush(h, a + b)
    return cost


def decode_tree_bits(tree: bytes, nbits: int):
    from blockparse import Bits, read_tree
    b = Bits(tree, 0, nbits)
    codes = read_tree(b)
    assert b.pos == nbits
    return codes


@pytest.mark.parametrize("seed", range(12))
def test_huffman_optimal_prefix_free_kraft(orc, seed):
    rng = np.random.default_rng(seed)
    freq = np.zeros(256, np.uint64)
    k = int(rng.integers(1, 257))
    idx = rng.choice(256, k, replace=False)
    freq[idx] = rng.integers(1, [2, 10, 1000, 100000][seed % 4], k)
    ln, code, tree, nbits = orc.huffman(freq)
    present = freq > 0
    assert (ln[~present] == -1).all()
    total = int(sum(int(freq[s]) * int(ln[s]) for s in range(256) if present[s]))
    assert total == optimal_cost([int(f) for f in freq])
    if k >= 2:
        assert sum(2.0 ** -int(ln[s]) for s in range(256) if present[s]) == 1.0
    else:
        assert ln[present].tolist() == [0]
    # tree: 10 n - 1 bits, and it yields exactly the codes
    assert nbits == 10 * k - 1
    codes = decode_tree_bits(tree.tobytes(), nbits)
    for cstr, s in codes.items():
        assert ln[s] == len(cstr)
        assert (format(int(code[s]), "b").zfill(len(cstr)) if len(cstr) else "") == cstr


def test_huffman_tie_break_fixture(orc):
    # equal weights: leaves sorted by symbol; leaf queue wins ties.
    # f(a=1)=f(b=2)=f(c=3)=f(d=4)=1: merge (1,2)->x, (3,4)->y, (x,y)->root
    freq = np.zeros(256, np.uint64)
    freq[[1, 2, 3, 4]] = 1
    ln, code, tree, nbits = orc.huffman(freq)
    assert [int(code[s]) for s in (1, 2, 3, 4)] == [0b00, 0b01, 0b10, 0b11]
    # f = 1,1,2: merge (1,2)->x(2); then the leaf 3 (weight 2) beats x on the tie
    freq[:] = 0
    freq[1], freq[2], freq[3] = 1, 1, 2
    ln, code, tree, nbits = orc.huffman(freq)
    assert (int(ln[3]), int(code[3])) == (1, 0)
    assert [(int(ln[s]), int(code[s])) for s in (1, 2)] == [(2, 0b10), (2, 0b11)]


# ------------------------------------------------------------ zero runs
def expand(tokens, czr):
    out = []
    for s, run in tokens:
        if s == czr:
            out.extend([czr] if run == 0 else [0] * run)
        else:
            assert run < 0
            out.append(s)
    return out


def test_zero_runs_bruteforce_roundtrip(orc):
    czr = 7
    for n in range(0, 10):
        for seq in itertools.product((0, czr, 3), repeat=n):
            for w in (2, 3):
                toks = orc.tokens(list(seq), czr, w)
                assert expand(toks, czr) == list(seq)
                M = 2 ** w - 1
                for (s, run), nxt in zip(toks, toks[1:] + [(None, None)]):
                    if s == czr:
                        assert 0 <= run <= M
                    if s == 0:                 # a literal zero is never next to another zero
                        assert nxt[0] != 0


def test_zero_runs_long_runs_split_greedily(orc):
    czr = 200
    for L in range(2, 40):
        toks = orc.tokens([0] * L + [5], czr, 2)
        runs = [r for s, r in toks if s == czr]
        assert runs == [3] * (L // 3) + ([L % 3] if L % 3 else [])


# --------------------------------------------------------- whole blocks
def random_block(rng, p, w, h, scale, sparsity):
    c = rng.laplace(0, scale, (p, h, w)).round().astype(np.int64)
    c[rng.random((p, h, w)) < sparsity] = 0
    return c


def block_cases():
    rng = np.random.default_rng(7)
    cases = []
    for p in (1, 3):
        for (w, h) in [(4, 4), (8, 4), (12, 20), (64, 64), (128, 128)]:
            for scale, sp in [(0.3, 0.9), (3, 0.5), (40, 0.1), (0.0, 1.0)]:
                cases.append(random_block(rng, p, w, h, scale, sp))
    # extremes
    cases.append(np.full((3, 8, 8), -(2 ** 14), np.int64))
    cases.append(np.full((1, 4, 4), 32767, np.int64))
    alt = np.zeros((1, 16, 16), np.int64)
    alt[0, ::2, ::2] = 1
    cases.append(alt)
    # tiny blocks: N_sym <= 4 symbols, so b = max(2, ceil(log2 N_sym)) = 2
    one = np.zeros((1, 4, 4), np.int64)
    one[0, 0, 0] = -1                       # d = 2, both planes kept: 4 symbols
    cases.append(one)
    one = np.zeros((1, 4, 4), np.int64)
    one[0, 2, 1] = 1                        # sign plane removed: 2 symbols
    cases.append(one)
    # dense halves beside zero halves: every byte value occurs in the kept planes (so C_zr occurs as
    # a literal, and Eq. 3's cost counts its literal tokens) next to long zero runs
    for frac in (0.5, 0.8, 0.95):
        c = rng.integers(-(1 << 10), 1 << 10, (3, 128, 128)).astype(np.int64)
        c[:, : int(128 * frac), :] = 0
        cases.append(c)
    # uniform symbols (C_zr occurs about 220 times as a literal) and one 4 x 8 hole, i.e. a run of 4
    # zero areas opening every plane: w = 2 wins only because the literal C_zr tokens are costed too
    # (without them, 3 counter bits and one pair per run would be cheaper)
    c = np.random.default_rng(3).integers(-1023, 1024, (3, 128, 128)).astype(np.int64)
    c[0, 0:4, 0:8] = 0
    cases.append(c)
    return cases


def expected_segments(orc, coef, removed, d):
    """Plane segment pl = the symbols of plane pl (Eq. 1 order, Eq. 2 values) of each kept type, the types
    in the block's order (HL, LH, HH), concatenated."""
    p, h, w = coef.shape
    n = w * h // 8
    segs = []
    for pl in range(d):
        seg = []
        for t in range(p):
            if removed[t][pl]:
                continue
            for k in range(pl * n, (pl + 1) * n):
                i, j, kp = orc.area_T(k, w, h)
                assert kp == pl
                seg.append(orc.area_symbol(coef[t], i, j, pl, d))
        segs.append(seg)
    return segs


def test_block_roundtrip_and_format(orc):
    for coef in block_cases():
        p, h, w = coef.shape
        data, st = orc.encode_block(coef)
        back = orc.decode_block(data, p, w, h)
        assert np.array_equal(back, coef)
        parsed = parse_block(data, p, w, h)
        if w * h * p <= 64 * 64 * 3 or coef.std() > 100:
            want = expected_segments(orc, coef, parsed["removed"], parsed["d"])
            got = [[] if pl is None else pl["symbols"] for pl in parsed["planes"]]
            assert got == want
        m = int(np.abs(coef).max())
        assert parsed["d"] == st["d"] == 1 + m.bit_length()
        # removed planes are exactly the all-zero (type, plane) symbol sets
        d = st["d"]
        for ty in range(p):
            a = coef[ty]
            for pl in range(d):
                plane = (a < 0) if pl == 0 else ((np.abs(a) >> (d - 1 - pl)) & 1).astype(bool)
                assert parsed["removed"][ty][pl] == int(not plane.any())
        if st["n_sym"] == 0:
            assert len(data) == (5 + p * d + 7) // 8
            continue
        # byte padding only at the end
        assert (parsed["total_bits"] + 7) // 8 == len(data)
        # t follows floor(log2(p w h / 8)) + 5 unless a segment needs more bits
        t0 = (p * w * h // 8).bit_length() - 1 + 5
        assert parsed["t"] == max(t0, max(s.bit_length() for s in parsed["seglen"]))
        check_block_properties(parsed, st, p, w, h)


def check_block_properties(parsed, st, p, w, h):
    czr, wb = parsed["czr"], parsed["w"]
    planes = [pl for pl in parsed["planes"] if pl is not None]
    raw = [s for pl in planes for s in pl["symbols"]]
    count = np.bincount(raw, minlength=256)
    # C_zr: least frequent of 1..255, smallest on ties
    assert count[czr] == count[1:].min()
    assert czr == 1 + int(np.argmin(count[1:]))
    # the code is optimal for the token frequencies it codes
    toks = [t for pl in planes for t in pl["tokens"]]
    tf = np.bincount([s for s, _, _ in toks], minlength=256)
    lens = {s: len(c) for c, s in parsed["codes"].items()}
    assert set(lens) == set(np.nonzero(tf)[0].tolist())
    assert sum(int(tf[s]) * lens[s] for s in lens) == optimal_cost(tf.tolist())
    # Eq. 3 (reading): w minimises (w + l) * pairs(w) over [2, b]
    runs = []
    for pl in planes:
        seq = pl["symbols"]
        i = 0
        while i < len(seq):
            if seq[i] == 0:
                j = i
                while j < len(seq) and seq[j] == 0:
                    j += 1
                if j - i >= 2:
                    runs.append(j - i)
                i = j
            else:
                i += 1
    b = max(2, (st["n_sym"] - 1).bit_length())
    assert st["b"] == b
    # l: C_zr's length in the provisional code, where each run counts once for C_zr and every other
    # symbol (isolated zeros and literal C_zr included) counts as itself.  Its lengths must be those of an
    # optimal code for exactly these counts (Huffman), and l the entry of C_zr.
    prov = np.zeros(256, np.int64)
    for pl in planes:
        seq, i = pl["symbols"], 0
        while i < len(seq):
            j = i
            while j < len(seq) and seq[j] == 0:
                j += 1
            if j - i >= 2:
                prov[czr] += 1
                i = j
            else:
                prov[seq[i]] += 1
                i += 1
    plen = np.array(st["prov_len"], np.int64)
    if (prov > 0).sum() >= 2:
        assert set(np.nonzero(plen)[0].tolist()) == set(np.nonzero(prov)[0].tolist())
        assert sum(2.0 ** -int(v) for v in plen[plen > 0]) == 1.0
        assert int((prov * plen).sum()) == optimal_cost(prov.tolist())
    assert st["l_prov"] == (int(plen[czr]) if prov[czr] > 0 else 0)
    costs = {wc: (wc + st["l_prov"]) * (int(count[czr]) + sum(-(-L // (2 ** wc - 1)) for L in runs))
             for wc in range(2, b + 1)}
    assert wb == min(costs, key=lambda k: (costs[k], k))
    # counters: every run token carries 1..2^w - 1 zeros
    for s, cnt, _ in toks:
        if s == czr:
            assert 0 <= cnt <= 2 ** wb - 1


def test_block_segments_decode_alone_and_lsb_drop(orc):
    rng = np.random.default_rng(11)
    for _ in range(10):
        coef = random_block(rng, 3, 32, 16, 20, 0.3)
        data, st = orc.encode_block(coef)
        d = st["d"]
        for drop in range(0, d + 1):
            back = orc.decode_block(data, 3, 32, 16, drop)
            mag = np.abs(coef) >> min(drop, d - 1) << min(drop, d - 1)
            assert np.array_equal(back, np.sign(coef) * mag)


def test_block_corrupt_input_is_an_error(orc):
    rng = np.random.default_rng(12)
    coef = random_block(rng, 3, 64, 64, 10, 0.2)
    data, st = orc.encode_block(coef)
    for cut in (1, 3, len(data) // 2, len(data) - 1):
        with pytest.raises(ValueError):
            orc.decode_block(data[:cut], 3, 64, 64)
