"""Independent reader of one compressed block, written from the documented
block layout (the paper's Fig. 3 fields in the order this codec fixes):

    d (5) | removed mask p*d (type-major, plane order) |
    [C_zr (8) | w (5) | t (5) | seektable d*t | preorder tree] | plane segments

Used by the tests to look inside the oracle's bytes (token streams, code
lengths, counters); it shares nothing with the oracle's C++ decoder.
"""
from __future__ import annotations


class Bits:
    def __init__(self, data: bytes, start: int = 0, end: int | None = None):
        self.data = data
        self.pos = start
        self.end = len(data) * 8 if end is None else end

    def get(self, n: int) -> int:
        v = 0
        for _ in range(n):
            if self.pos >= self.end:
                raise ValueError("read past end")
            byte = self.data[self.pos >> 3]
            v = (v << 1) | ((byte >> (7 - (self.pos & 7))) & 1)
            self.pos += 1
        return v


def read_tree(b: Bits, prefix: str = "", codes=None, depth: int = 0):
    if codes is None:
        codes = {}
    if depth > 32:
        raise ValueError("tree too deep")
    if b.get(1):
        codes[prefix] = b.get(8)
    else:
        read_tree(b, prefix + "0", codes, depth + 1)
        read_tree(b, prefix + "1", codes, depth + 1)
    return codes


def parse_block(data: bytes, p: int, w: int, h: int):
    n = w * h // 8
    b = Bits(data)
    d = b.get(5)
    removed = [[b.get(1) for _ in range(d)] for _ in range(p)]
    out = {"d": d, "removed": removed, "header_bits": None, "planes": [None] * d}
    if all(all(r) for r in removed):
        out["header_bits"] = b.pos
        return out
    czr, wbits, t = b.get(8), b.get(5), b.get(5)
    seglen = [b.get(t) for _ in range(d)]
    tree_start = b.pos
    codes = read_tree(b)
    out.update(czr=czr, w=wbits, t=t, seglen=seglen, codes=codes, tree_bits=b.pos - tree_start)
    out["header_bits"] = b.pos
    start = b.pos
    for pl in range(d):
        kept = sum(1 for ty in range(p) if not removed[ty][pl])
        if kept == 0:
            assert seglen[pl] == 0
            continue
        sb = Bits(data, start, start + seglen[pl])
        toks, syms = [], []
        while len(syms) < kept * n:
            if "" in codes:
                s = codes[""]
                code = ""
            else:
                code = ""
                while code not in codes:
                    code += "1" if sb.get(1) else "0"
                s = codes[code]
            if s == czr:
                cnt = sb.get(wbits)
                toks.append((s, cnt, code))
                syms.extend([czr] if cnt == 0 else [0] * cnt)
            else:
                toks.append((s, None, code))
                syms.append(s)
        assert sb.pos == sb.end, "segment length in seektable does not match its tokens"
        out["planes"][pl] = {"tokens": toks, "symbols": syms, "kept_types": kept}
        start += seglen[pl]
    out["total_bits"] = start
    return out
