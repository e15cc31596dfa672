// isx_oracle.cpp — plain, slow CPU reference of the codec of Hulsken,
// "Fast Compression Method for Medical Images on the Web" (2020).
//
// TEST INFRASTRUCTURE ONLY.  This file defines the exact bitstream and pixel
// results that the GPU library must reproduce.  Only the test suite, the
// smoke check and the benchmark's CPU-baseline leg may load it; the product
// path never calls it.  It shares no code, header or table with the CUDA
// library (paper_2005_08713_gb300/csrc).
//
// Every step follows the paper in its own order (Fig. 1, Fig. 2 a-e):
//   colour transform -> recursive 5/3 wavelet -> (quantisation) ->
//   128x128 blocks -> SMR bitplanes -> 4x2 areas in snake order (Eq. 1) ->
//   area symbols (Eq. 2) -> empty-plane removal -> zero runs (Eq. 3) ->
//   Huffman -> block container (Fig. 3).
// Where the paper is silent or garbled the reading used is stated at the
// function; the readings are collected in the design notes of the repo.
//
// All integer arithmetic is int64_t; floor division is written out.
// "parity unpinned" functions (no paper example exists): the Eq. 1 area
// order, the block header field order (Fig. 3 is missing), the Huffman
// tie-break shape, the Eq. 3 cost reading and the 2-D lifting order
// (columns, then rows: integer lifting does not commute, and the paper
// does not say).  Their pins are invariants (bijection, round trip,
// optimal length), not paper bytes.

#include <cstdint>
#include <cstring>
#include <cstdlib>
#include <vector>
#include <algorithm>
#include <thread>
#include <atomic>

namespace {

// ---------------------------------------------------------------- helpers

int64_t floordiv(int64_t a, int64_t b) {  // b > 0; rounds toward -infinity
  int64_t q = a / b;
  if ((a % b) != 0 && (a < 0)) q -= 1;
  return q;
}

int64_t ceildiv(int64_t a, int64_t b) { return (a + b - 1) / b; }  // a >= 0, b > 0

int bitlen(uint64_t v) {  // number of bits needed to write v (bitlen(0) = 0)
  int n = 0;
  while (v) { n++; v >>= 1; }
  return n;
}

// MSB-first bit writer: the block is one big-endian bit string (Sec. 4:
// counters are big endian, header fields are not byte aligned).
struct BitWriter {
  std::vector<uint8_t> bytes;
  uint64_t nbits = 0;
  void put(uint64_t value, int n) {  // writes the n low bits of value, MSB first
    for (int i = n - 1; i >= 0; --i) {
      uint64_t bit = (value >> i) & 1u;
      if (nbits % 8 == 0) bytes.push_back(0);
      if (bit) bytes.back() |= (uint8_t)(0x80u >> (nbits % 8));
      nbits++;
    }
  }
};

struct BitReader {
  const uint8_t* data;
  uint64_t nbits_total;
  uint64_t pos;
  bool overrun = false;
  uint64_t get(int n) {
    uint64_t v = 0;
    for (int i = 0; i < n; ++i) {
      uint64_t bit = 0;
      if (pos < nbits_total) bit = (data[pos / 8] >> (7 - pos % 8)) & 1u;
      else overrun = true;
      v = (v << 1) | bit;
      pos++;
    }
    return v;
  }
};

// ------------------------------------------------- colour transform (Fig. 1)
// The paper names only an "(optional) colorspace transformation" (Sec. 3).
// Reading: the reversible colour transform of JPEG 2000 (ISO/IEC 15444-1
// Annex G), chosen because the paper reuses JPEG 2000's quantisation.
//   Y = floor((R + 2G + B) / 4),  Cb = B - G,  Cr = R - G
void rct_forward(int64_t R, int64_t G, int64_t B, int64_t* Y, int64_t* Cb, int64_t* Cr) {
  *Y = floordiv(R + 2 * G + B, 4);
  *Cb = B - G;
  *Cr = R - G;
}
//   G = Y - floor((Cb + Cr) / 4),  R = Cr + G,  B = Cb + G
void rct_inverse(int64_t Y, int64_t Cb, int64_t Cr, int64_t* R, int64_t* G, int64_t* B) {
  *G = Y - floordiv(Cb + Cr, 4);
  *R = Cr + *G;
  *B = Cb + *G;
}

// The alternative reversible colour transform the build also offers:
// YCoCg-R (Malvar and Sullivan, "YCoCg-R: A Color Space with RGB
// Reversibility and Low Dynamic Range", JVT-I014, 2003), two lifting steps
// per chroma pair:
//   Co = R - B,  t = B + floor(Co / 2),  Cg = G - t,  Y = t + floor(Cg / 2)
void ycocg_forward(int64_t R, int64_t G, int64_t B, int64_t* Y, int64_t* Co, int64_t* Cg) {
  *Co = R - B;
  const int64_t t = B + floordiv(*Co, 2);
  *Cg = G - t;
  *Y = t + floordiv(*Cg, 2);
}
//   t = Y - floor(Cg / 2),  G = Cg + t,  B = t - floor(Co / 2),  R = B + Co
void ycocg_inverse(int64_t Y, int64_t Co, int64_t Cg, int64_t* R, int64_t* G, int64_t* B) {
  const int64_t t = Y - floordiv(Cg, 2);
  *G = Cg + t;
  *B = t - floordiv(Co, 2);
  *R = *B + Co;
}

// ------------------------------------------- 5/3 Le Gall integer lifting (Sec. 4)
// Reading: the reversible 5/3 of ISO/IEC 15444-1 Annex F with whole-sample
// symmetric extension, even-indexed samples low-pass:
//   predict  d[n] = x[2n+1] - floor((x[2n] + x[2n+2]) / 2)
//   update   s[n] = x[2n]   + floor((d[n-1] + d[n] + 2) / 4)
// The signal is extended by mirroring about its first and last sample, so
// a value needed outside [0, N) is the one at the mirrored position; the
// high-pass sequence inherits the same mirror (d at odd position q equals d
// at the mirror of q).  N -> ceil(N/2) low, floor(N/2) high; N = 1 passes.
int64_t mirror(int64_t i, int64_t n) {  // whole-sample symmetric index into [0, n)
  if (n == 1) return 0;
  int64_t period = 2 * (n - 1);
  i %= period;
  if (i < 0) i += period;
  if (i >= n) i = period - i;
  return i;
}

void lift53_forward(const int64_t* x, int64_t n, int64_t* low, int64_t* high) {
  if (n <= 0) return;
  if (n == 1) { low[0] = x[0]; return; }
  auto X = [&](int64_t i) { return x[mirror(i, n)]; };
  int64_t nh = n / 2, nl = (n + 1) / 2;
  // predict: every odd position of the (extended) signal
  for (int64_t k = 0; k < nh; ++k)
    high[k] = X(2 * k + 1) - floordiv(X(2 * k) + X(2 * k + 2), 2);
  auto D = [&](int64_t k) {  // d at odd position 2k+1, extended by the mirror
    int64_t q = mirror(2 * k + 1, n);
    return high[(q - 1) / 2];
  };
  // update: every even position
  for (int64_t k = 0; k < nl; ++k)
    low[k] = X(2 * k) + floordiv(D(k - 1) + D(k) + 2, 4);
}

void lift53_inverse(const int64_t* low, const int64_t* high, int64_t n, int64_t* x) {
  if (n <= 0) return;
  if (n == 1) { x[0] = low[0]; return; }
  int64_t nh = n / 2, nl = (n + 1) / 2;
  auto D = [&](int64_t k) {
    int64_t q = mirror(2 * k + 1, n);
    return high[(q - 1) / 2];
  };
  // undo update: even positions
  for (int64_t k = 0; k < nl; ++k)
    x[2 * k] = low[k] - floordiv(D(k - 1) + D(k) + 2, 4);
  // undo predict: odd positions (even neighbours are final now)
  auto X = [&](int64_t i) { return x[mirror(i, n)]; };
  for (int64_t k = 0; k < nh; ++k)
    x[2 * k + 1] = high[k] + floordiv(X(2 * k) + X(2 * k + 2), 2);
}

// ------------------------------------------------ recursive 2-D wavelet (Fig. 1)
// Reading (paper silent on 2-D order): per level, 1-D lifting down every
// column, then along every row, of the current LL, as in JPEG 2000's
// 2D_SD.  Result in Mallat layout: after a level on a w x h region the
// top-left ceil(w/2) x ceil(h/2) is LL, top-right HL (high horizontally,
// low vertically), bottom-left LH, bottom-right HH.  Recurse on LL.
// plane: row-major, stride `stride`.
void dwt2_forward(int64_t* plane, int64_t stride, int64_t w, int64_t h, int levels) {
  std::vector<int64_t> line, lo, hi;
  int64_t cw = w, ch = h;
  for (int l = 0; l < levels; ++l) {
    // columns
    line.resize(ch); lo.resize(ch); hi.resize(ch);
    for (int64_t c = 0; c < cw; ++c) {
      for (int64_t r = 0; r < ch; ++r) line[r] = plane[r * stride + c];
      lift53_forward(line.data(), ch, lo.data(), hi.data());
      int64_t nl = (ch + 1) / 2;
      for (int64_t r = 0; r < nl; ++r) plane[r * stride + c] = lo[r];
      for (int64_t r = 0; r < ch / 2; ++r) plane[(nl + r) * stride + c] = hi[r];
    }
    // rows
    line.resize(cw); lo.resize(cw); hi.resize(cw);
    for (int64_t r = 0; r < ch; ++r) {
      for (int64_t c = 0; c < cw; ++c) line[c] = plane[r * stride + c];
      lift53_forward(line.data(), cw, lo.data(), hi.data());
      int64_t nl = (cw + 1) / 2;
      for (int64_t c = 0; c < nl; ++c) plane[r * stride + c] = lo[c];
      for (int64_t c = 0; c < cw / 2; ++c) plane[r * stride + nl + c] = hi[c];
    }
    cw = (cw + 1) / 2;
    ch = (ch + 1) / 2;
  }
}

// Inverse of dwt2_forward on the w x h region (levels applied to it).
void dwt2_inverse(int64_t* plane, int64_t stride, int64_t w, int64_t h, int levels) {
  std::vector<int64_t> dims_w(levels + 1), dims_h(levels + 1);
  dims_w[0] = w; dims_h[0] = h;
  for (int l = 1; l <= levels; ++l) {
    dims_w[l] = (dims_w[l - 1] + 1) / 2;
    dims_h[l] = (dims_h[l - 1] + 1) / 2;
  }
  std::vector<int64_t> line, lo, hi;
  for (int l = levels; l >= 1; --l) {
    int64_t cw = dims_w[l - 1], ch = dims_h[l - 1];
    // rows first (reverse of the forward order)
    line.resize(cw); lo.resize(cw); hi.resize(cw);
    for (int64_t r = 0; r < ch; ++r) {
      int64_t nl = (cw + 1) / 2;
      for (int64_t c = 0; c < nl; ++c) lo[c] = plane[r * stride + c];
      for (int64_t c = 0; c < cw / 2; ++c) hi[c] = plane[r * stride + nl + c];
      lift53_inverse(lo.data(), hi.data(), cw, line.data());
      for (int64_t c = 0; c < cw; ++c) plane[r * stride + c] = line[c];
    }
    line.resize(ch); lo.resize(ch); hi.resize(ch);
    for (int64_t c = 0; c < cw; ++c) {
      int64_t nl = (ch + 1) / 2;
      for (int64_t r = 0; r < nl; ++r) lo[r] = plane[r * stride + c];
      for (int64_t r = 0; r < ch / 2; ++r) hi[r] = plane[(nl + r) * stride + c];
      lift53_inverse(lo.data(), hi.data(), ch, line.data());
      for (int64_t r = 0; r < ch; ++r) plane[r * stride + c] = line[r];
    }
  }
}

// ------------------------------------------------------ quantisation (Sec. 3)
// "the same image quantization methods as in JPEG2000": dead-zone scalar
// quantiser with an integer step Delta = 2^q;  q = sign(c) floor(|c|/Delta).
// Reconstruction at the bin midpoint: c' = sign(q) (|q| Delta + floor(Delta/2)),
// 0 for q = 0.  Delta = 1 is the identity (lossless).
int64_t quantise(int64_t c, int64_t delta) {
  int64_t m = c < 0 ? -c : c;
  int64_t q = m / delta;
  return c < 0 ? -q : q;
}
int64_t dequantise(int64_t q, int64_t delta) {
  if (q == 0) return 0;
  int64_t m = (q < 0 ? -q : q) * delta + delta / 2;
  return q < 0 ? -m : m;
}

// ---------------------------------------------------- area order T(k) (Eq. 1)
// Printed Eq. 1 is garbled.  Reading, for a w x h block (w, h multiples of
// 4) of bit depth d, with k' = k mod (wh/8):
//   plane index p = floor(8k / wh)     (p = 0 sign plane, then magnitude
//                                       MSB..LSB: "sign first, then MSB down")
//   row    i = 4 floor(2k'/w) + 2 (k mod 2)
//   column j = 4 (floor(k/2) mod (w/4))          (as printed)
// i.e. the two vertically stacked 4x2 areas of a 4-column group, then the
// next group to the right, then the next 4-row band.
void area_T(int64_t k, int64_t w, int64_t h, int64_t* i, int64_t* j, int64_t* p) {
  int64_t n = w * h / 8;
  int64_t kk = k % n;
  *p = (8 * k) / (w * h);
  *i = 4 * ((2 * kk) / w) + 2 * (k % 2);
  *j = 4 * ((k / 2) % (w / 4));
}

// bit of coefficient value c in serialised plane p of a block of depth d:
// p = 0 is the sign (1 for negative), p >= 1 is magnitude bit d-1-p.
int plane_bit(int64_t c, int64_t p, int64_t d) {
  if (p == 0) return c < 0 ? 1 : 0;
  int64_t m = c < 0 ? -c : c;
  return (int)((m >> (d - 1 - p)) & 1);
}

// ------------------------------------------------------ area symbol (Eq. 2)
// S_k = sum_{m=i..i+1} sum_{n=j..j+3} B(m,n,b) 2^{(n-j) + 4(m-i)}
// (the explicit equation is followed; the caption's "clockwise" wording
// would reverse the lower row).
// coef: row-major w-wide block of one coefficient type.
int area_symbol(const int64_t* coef, int64_t w, int64_t i, int64_t j, int64_t p, int64_t d) {
  int s = 0;
  for (int64_t m = i; m <= i + 1; ++m)
    for (int64_t n = j; n <= j + 3; ++n)
      s += plane_bit(coef[m * w + n], p, d) << ((n - j) + 4 * (m - i));
  return s;
}

// ------------------------------------------------------------- Huffman code
// "created as normal" (Sec. 4).  Reading: the two-queue construction.
// Leaves with f > 0 sorted ascending by (f, symbol) form queue 1; merged
// nodes join queue 2 in creation order.  Each merge takes the lighter front
// twice (on equal weight queue 1, the leaves, first); the first node taken
// becomes the left child (bit 0), the second the right child (bit 1).
struct HuffNode { uint64_t weight; int left, right; int symbol; };  // symbol >= 0 for leaves

struct HuffCode {
  int n_leaves = 0;
  int root = -1;
  std::vector<HuffNode> nodes;
  uint32_t code[256];
  int len[256];
};

HuffCode huffman_build(const uint64_t* freq) {
  HuffCode hc;
  for (int s = 0; s < 256; ++s) { hc.code[s] = 0; hc.len[s] = -1; }
  std::vector<int> leaves;
  for (int s = 0; s < 256; ++s)
    if (freq[s] > 0) {
      hc.nodes.push_back({freq[s], -1, -1, s});
      leaves.push_back((int)hc.nodes.size() - 1);
    }
  hc.n_leaves = (int)leaves.size();
  if (hc.n_leaves == 0) return hc;
  std::stable_sort(leaves.begin(), leaves.end(), [&](int a, int b) {
    if (hc.nodes[a].weight != hc.nodes[b].weight) return hc.nodes[a].weight < hc.nodes[b].weight;
    return hc.nodes[a].symbol < hc.nodes[b].symbol;
  });
  std::vector<int> merged;
  size_t qa = 0, qb = 0;
  auto take = [&]() {
    bool from_leaves;
    if (qa < leaves.size() && qb < merged.size())
      from_leaves = hc.nodes[leaves[qa]].weight <= hc.nodes[merged[qb]].weight;
    else
      from_leaves = qa < leaves.size();
    return from_leaves ? leaves[qa++] : merged[qb++];
  };
  int remaining = hc.n_leaves;
  while (remaining > 1) {
    int a = take();
    int b = take();
    hc.nodes.push_back({hc.nodes[a].weight + hc.nodes[b].weight, a, b, -1});
    merged.push_back((int)hc.nodes.size() - 1);
    remaining--;
  }
  hc.root = hc.n_leaves == 1 ? leaves[0] : merged.back();
  // codes: walk from the root, left = 0, right = 1; a lone leaf has length 0
  std::vector<std::pair<int, std::pair<uint32_t, int>>> stack;
  stack.push_back({hc.root, {0u, 0}});
  while (!stack.empty()) {
    auto top = stack.back(); stack.pop_back();
    const HuffNode& nd = hc.nodes[top.first];
    if (nd.symbol >= 0) {
      hc.code[nd.symbol] = top.second.first;
      hc.len[nd.symbol] = top.second.second;
    } else {
      stack.push_back({nd.left, {top.second.first << 1, top.second.second + 1}});
      stack.push_back({nd.right, {(top.second.first << 1) | 1u, top.second.second + 1}});
    }
  }
  return hc;
}

// Fig. 3: tree stored recursively, 0 = internal node, 1 + 8-bit symbol = leaf.
void huffman_write_tree(const HuffCode& hc, int node, BitWriter& bw) {
  const HuffNode& nd = hc.nodes[node];
  if (nd.symbol >= 0) { bw.put(1, 1); bw.put((uint64_t)nd.symbol, 8); return; }
  bw.put(0, 1);
  huffman_write_tree(hc, nd.left, bw);
  huffman_write_tree(hc, nd.right, bw);
}

// Decoding tree as read back: nodes with children, leaves with symbols.
struct DecTree {
  std::vector<int> left, right, symbol;
  bool bad = false;
};
int read_tree(BitReader& br, DecTree& t, int depth) {
  if (depth > 32 || t.symbol.size() > 600 || br.overrun) { t.bad = true; return -1; }
  int id = (int)t.symbol.size();
  t.left.push_back(-1); t.right.push_back(-1); t.symbol.push_back(-1);
  if (br.get(1)) {
    t.symbol[id] = (int)br.get(8);
  } else {
    int l = read_tree(br, t, depth + 1);
    int r = read_tree(br, t, depth + 1);
    t.left[id] = l; t.right[id] = r;
  }
  return id;
}

// ------------------------------------------------------------ block coding
// A coefficient block (Fig. 3): p = 1 (LL) or p = 3 types (HL, LH, HH, in
// that order), each w x h after zero padding to multiples of 4, bit depth d.
struct Block {
  int p = 1;
  int64_t w = 4, h = 4;
  std::vector<int64_t> coef[3];  // row-major h x w, zero padded
};

// Block bit depth: d = 1 + bitlen(max |c|)  (sign plane + magnitude planes).
int block_depth(const Block& b) {
  uint64_t mx = 0;
  for (int t = 0; t < b.p; ++t)
    for (int64_t v : b.coef[t]) mx = std::max<uint64_t>(mx, (uint64_t)(v < 0 ? -v : v));
  return 1 + bitlen(mx);
}

// Zero-run reading (Sec. 4, Fig. 2e): inside one plane segment, a maximal
// stretch of >= 2 zero symbols is a run; C_zr followed by a w-bit counter
// holding a length 1..2^w-1; a run longer than 2^w-1 is a sequence of
// pairs, full ones first.  A literal C_zr is C_zr with counter 0.  An
// isolated zero is the literal symbol 0.
struct Token { int symbol; int64_t run; };  // run < 0: literal symbol; run >= 1: zero-run pair

// Splits a plane segment into literals and maximal zero runs (run lengths >= 2).
struct SegmentRuns {
  std::vector<int> literals_and_runs_kind;  // 0 literal, 1 run
  std::vector<int64_t> value;               // symbol for literal, length for run
};
SegmentRuns find_runs(const std::vector<int>& seg) {
  SegmentRuns r;
  size_t i = 0;
  while (i < seg.size()) {
    if (seg[i] == 0) {
      size_t j = i;
      while (j < seg.size() && seg[j] == 0) ++j;
      if (j - i >= 2) { r.literals_and_runs_kind.push_back(1); r.value.push_back((int64_t)(j - i)); }
      else { r.literals_and_runs_kind.push_back(0); r.value.push_back(0); }
      i = j;
    } else {
      r.literals_and_runs_kind.push_back(0); r.value.push_back(seg[i]);
      ++i;
    }
  }
  return r;
}

std::vector<Token> tokens_of(const SegmentRuns& r, int czr, int w) {
  std::vector<Token> out;
  int64_t M = ((int64_t)1 << w) - 1;
  for (size_t e = 0; e < r.value.size(); ++e) {
    if (r.literals_and_runs_kind[e] == 0) {
      int s = (int)r.value[e];
      out.push_back({s, s == czr ? 0 : -1});
    } else {
      int64_t L = r.value[e];
      while (L > 0) {
        int64_t n = L >= M ? M : L;
        out.push_back({czr, n});
        L -= n;
      }
    }
  }
  return out;
}

struct EncodeStats {  // exposed for the pins (Eq. 3 choice, Huffman)
  int d, czr, w, t, b, l_prov, n_kept_planes;
  int prov_len[256];    // code lengths of the provisional code of Eq. 3's l (0 = symbol absent)
  int64_t n_sym;
};

std::vector<uint8_t> encode_block(const Block& blk, EncodeStats* st) {
  const int p = blk.p;
  const int64_t w = blk.w, h = blk.h, n = w * h / 8;
  const int d = block_depth(blk);
  // Step c/d (Fig. 2): areas in Eq. 1 order, symbols by Eq. 2, per type.
  std::vector<std::vector<int>> sym(p, std::vector<int>((size_t)(d * n)));
  for (int t = 0; t < p; ++t)
    for (int64_t k = 0; k < d * n; ++k) {
      int64_t i, j, pl;
      area_T(k, w, h, &i, &j, &pl);
      sym[t][k] = area_symbol(blk.coef[t].data(), w, i, j, pl, d);
    }
  // Empty bitplane removal: a plane of one type whose symbols are all zero.
  std::vector<std::vector<int>> removed(p, std::vector<int>(d, 1));
  for (int t = 0; t < p; ++t)
    for (int pl = 0; pl < d; ++pl)
      for (int64_t k = 0; k < n; ++k)
        if (sym[t][pl * n + k] != 0) { removed[t][pl] = 0; break; }
  // Plane segment pl = kept types' symbols of plane pl, types in order.
  std::vector<std::vector<int>> seg(d);
  int64_t n_sym = 0;
  for (int pl = 0; pl < d; ++pl)
    for (int t = 0; t < p; ++t)
      if (!removed[t][pl])
        for (int64_t k = 0; k < n; ++k) seg[pl].push_back(sym[t][pl * n + k]);
  for (int pl = 0; pl < d; ++pl) n_sym += (int64_t)seg[pl].size();

  BitWriter bw;
  bw.put((uint64_t)d, 5);
  for (int t = 0; t < p; ++t)
    for (int pl = 0; pl < d; ++pl) bw.put((uint64_t)removed[t][pl], 1);
  if (st) {
    st->d = d; st->n_sym = n_sym; st->czr = -1; st->w = -1; st->t = -1; st->b = -1; st->l_prov = -1;
    for (int s = 0; s < 256; ++s) st->prov_len[s] = 0;
  }
  if (n_sym == 0) return bw.bytes;  // nothing kept: mask only

  // Zero-run symbol: least frequent of 1..255 among the kept symbols,
  // ties to the smallest value (a symbol that never occurs wins).
  uint64_t count[256] = {0};
  for (int pl = 0; pl < d; ++pl)
    for (int s : seg[pl]) count[s]++;
  int czr = 1;
  for (int s = 2; s < 256; ++s)
    if (count[s] < count[czr]) czr = s;
  std::vector<SegmentRuns> runs(d);
  for (int pl = 0; pl < d; ++pl) runs[pl] = find_runs(seg[pl]);

  // Eq. 3 reading: w minimises the exact cost of the C_zr tokens,
  //   cost(w) = (w + l) * (sum_runs ceil(L / (2^w - 1)) + count(C_zr)),
  // over w in [2, b], b = max(2, ceil(log2 N_sym)), ties to the smallest w;
  // l = C_zr's code length in a provisional Huffman code in which every
  // run counts once for C_zr.
  uint64_t prov[256] = {0};
  for (int pl = 0; pl < d; ++pl)
    for (size_t e = 0; e < runs[pl].value.size(); ++e) {
      if (runs[pl].literals_and_runs_kind[e] == 0) prov[runs[pl].value[e]]++;
      else prov[czr]++;
    }
  HuffCode hprov = huffman_build(prov);
  int l = prov[czr] > 0 ? hprov.len[czr] : 0;
  if (st)
    for (int s = 0; s < 256; ++s) st->prov_len[s] = hprov.len[s] > 0 ? hprov.len[s] : 0;
  int b = 0;
  while (((int64_t)1 << b) < n_sym) ++b;  // ceil(log2 n_sym)
  if (b < 2) b = 2;
  int best_w = 2;
  uint64_t best_cost = UINT64_MAX;
  for (int wc = 2; wc <= b; ++wc) {
    int64_t M = ((int64_t)1 << wc) - 1;
    uint64_t pairs = count[czr];
    for (int pl = 0; pl < d; ++pl)
      for (size_t e = 0; e < runs[pl].value.size(); ++e)
        if (runs[pl].literals_and_runs_kind[e] == 1) pairs += (uint64_t)ceildiv(runs[pl].value[e], M);
    uint64_t cost = (uint64_t)(wc + l) * pairs;
    if (cost < best_cost) { best_cost = cost; best_w = wc; }
  }
  const int w_bits = best_w;

  // Final Huffman code over the tokens (runs expanded into their pairs).
  std::vector<std::vector<Token>> toks(d);
  uint64_t freq[256] = {0};
  for (int pl = 0; pl < d; ++pl) {
    toks[pl] = tokens_of(runs[pl], czr, w_bits);
    for (const Token& tk : toks[pl]) freq[tk.symbol]++;
  }
  HuffCode hc = huffman_build(freq);

  // Plane segments as bit strings.
  std::vector<BitWriter> segbits(d);
  for (int pl = 0; pl < d; ++pl)
    for (const Token& tk : toks[pl]) {
      segbits[pl].put(hc.code[tk.symbol], hc.len[tk.symbol]);
      if (tk.symbol == czr) segbits[pl].put((uint64_t)tk.run, w_bits);
    }
  // Seektable (Fig. 3): d entries of t bits, entry = bit length of plane
  // segment pl (0 for a removed plane); t = floor(log2(p w h / 8)) + 5,
  // raised only if a segment length does not fit.
  int t_bits = bitlen((uint64_t)(p * w * h / 8)) - 1 + 5;
  for (int pl = 0; pl < d; ++pl) t_bits = std::max(t_bits, bitlen(segbits[pl].nbits));

  bw.put((uint64_t)czr, 8);
  bw.put((uint64_t)w_bits, 5);
  bw.put((uint64_t)t_bits, 5);
  for (int pl = 0; pl < d; ++pl) bw.put(segbits[pl].nbits, t_bits);
  huffman_write_tree(hc, hc.root, bw);
  for (int pl = 0; pl < d; ++pl) {
    BitReader br{segbits[pl].bytes.data(), segbits[pl].nbits, 0};
    uint64_t left = segbits[pl].nbits;
    while (left > 0) {
      int take = left > 32 ? 32 : (int)left;
      bw.put(br.get(take), take);
      left -= (uint64_t)take;
    }
  }
  if (st) { st->czr = czr; st->w = w_bits; st->t = t_bits; st->b = b; st->l_prov = l; }
  return bw.bytes;
}

// Decode a block; planes pl >= d - drop (the `drop` least significant
// magnitude planes) are discarded (Sec. 4: reconstruction "by discarding an
// arbitrary number of the least significant bits").  Returns 0 or -1.
int decode_block(const uint8_t* data, int64_t size, Block& blk, int drop) {
  const int p = blk.p;
  const int64_t w = blk.w, h = blk.h, n = w * h / 8;
  for (int t = 0; t < p; ++t) blk.coef[t].assign((size_t)(w * h), 0);
  BitReader br{data, (uint64_t)size * 8, 0};
  int d = (int)br.get(5);
  if (d < 1) return -1;
  std::vector<std::vector<int>> removed(p, std::vector<int>(d));
  bool any_kept = false;
  for (int t = 0; t < p; ++t)
    for (int pl = 0; pl < d; ++pl) { removed[t][pl] = (int)br.get(1); any_kept |= !removed[t][pl]; }
  if (br.overrun) return -1;
  if (!any_kept) return 0;
  int czr = (int)br.get(8);
  int w_bits = (int)br.get(5);
  int t_bits = (int)br.get(5);
  std::vector<uint64_t> seglen(d);
  for (int pl = 0; pl < d; ++pl) seglen[pl] = br.get(t_bits);
  DecTree tree;
  read_tree(br, tree, 0);
  if (tree.bad || br.overrun) return -1;
  std::vector<uint64_t> segstart(d);
  uint64_t pos = br.pos;
  for (int pl = 0; pl < d; ++pl) { segstart[pl] = pos; pos += seglen[pl]; }
  if (pos > (uint64_t)size * 8) return -1;
  int keep_planes = d - drop;
  if (keep_planes < 1) keep_planes = 1;  // the sign plane is always kept
  // magnitudes and signs accumulated from the planes that are decoded
  std::vector<std::vector<int>> symbols(p, std::vector<int>((size_t)(d * n), 0));
  for (int pl = 0; pl < keep_planes; ++pl) {
    int kept_types = 0;
    for (int t = 0; t < p; ++t) kept_types += !removed[t][pl];
    if (kept_types == 0) continue;
    // each segment is decoded on its own from its seektable start
    BitReader sr{data, segstart[pl] + seglen[pl], segstart[pl]};
    std::vector<int> seg;
    int64_t need = kept_types * n;
    while ((int64_t)seg.size() < need) {
      int node = 0;
      int guard = 0;
      while (tree.symbol[node] < 0) {
        node = sr.get(1) ? tree.right[node] : tree.left[node];
        if (node < 0 || ++guard > 32) return -1;
      }
      int s = tree.symbol[node];
      if (s == czr) {
        int64_t cnt = (int64_t)sr.get(w_bits);
        if (cnt == 0) seg.push_back(czr);
        else for (int64_t e = 0; e < cnt; ++e) seg.push_back(0);
      } else {
        seg.push_back(s);
      }
      if (sr.overrun) return -1;
    }
    if ((int64_t)seg.size() != need) return -1;
    int64_t pos_in_seg = 0;
    for (int t = 0; t < p; ++t) {
      if (removed[t][pl]) continue;
      for (int64_t k = 0; k < n; ++k) symbols[t][pl * n + k] = seg[pos_in_seg++];
    }
  }
  // Invert Eq. 1 / Eq. 2: place each symbol's bits back.
  for (int t = 0; t < p; ++t) {
    std::vector<int64_t> mag((size_t)(w * h), 0);
    std::vector<int> neg((size_t)(w * h), 0);
    for (int64_t k = 0; k < d * n; ++k) {
      int64_t i, j, pl;
      area_T(k, w, h, &i, &j, &pl);
      int s = symbols[t][k];
      for (int64_t m = i; m <= i + 1; ++m)
        for (int64_t c = j; c <= j + 3; ++c) {
          int bit = (s >> ((c - j) + 4 * (m - i))) & 1;
          if (!bit) continue;
          if (pl == 0) neg[m * w + c] = 1;
          else mag[m * w + c] |= (int64_t)1 << (d - 1 - pl);
        }
    }
    for (int64_t e = 0; e < w * h; ++e) blk.coef[t][e] = neg[e] ? -mag[e] : mag[e];
  }
  return 0;
}

// ------------------------------------------------------- tile container
// Byte layout of a tile stream (the paper defines only the block, Fig. 3):
//   0  'I' 'S' 'X' '1'
//   4  u16 width        6  u16 height
//   8  u8 channels      9  u8 bits     10 u8 levels
//  11  u8 colour transform of channels 0..2 (0 none, 1 RCT, 2 YCoCg-R)
//  12  u32 n_blocks
//  16  u8 qstep_log2[16]   (index l-1 for level l, index `levels` for the LL)
//  32  u32 block_end[n_blocks]  (cumulative byte ends, relative to the block data)
//  32 + 4 n_blocks: block data, each block byte aligned.
// All multi-byte fields little endian.
// Block order: channel-major; per channel the LL blocks, then the
// high-pass blocks of level L, L-1, ..., 1; blocks of one subband in raster
// order of 128 x 128 cells anchored at the subband origin.
struct TileInfo {
  int w, h, C, bits, L, ct;
  uint8_t q[16];
};

struct BlockRef { int c; int level; /* 0 = LL */ int by, bx; };

int64_t level_dim(int64_t n, int l) {  // size of LL_l along one axis
  for (int i = 0; i < l; ++i) n = (n + 1) / 2;
  return n;
}

std::vector<BlockRef> tile_blocks(const TileInfo& ti) {
  std::vector<BlockRef> out;
  for (int c = 0; c < ti.C; ++c) {
    int64_t lw = level_dim(ti.w, ti.L), lh = level_dim(ti.h, ti.L);
    for (int by = 0; by < ceildiv(lh, 128); ++by)
      for (int bx = 0; bx < ceildiv(lw, 128); ++bx) out.push_back({c, 0, by, bx});
    for (int l = ti.L; l >= 1; --l) {
      int64_t gw = level_dim(ti.w, l), gh = level_dim(ti.h, l);  // grid over max type extent
      for (int by = 0; by < ceildiv(gh, 128); ++by)
        for (int bx = 0; bx < ceildiv(gw, 128); ++bx) out.push_back({c, l, by, bx});
    }
  }
  return out;
}

// Subband rectangle inside the Mallat plane: type 0 = LL_L (level 0 ref),
// for a level l: type 0 HL, 1 LH, 2 HH.
void subband_rect(const TileInfo& ti, int level, int type, int64_t* x, int64_t* y, int64_t* sw, int64_t* sh) {
  if (level == 0) {
    *x = 0; *y = 0; *sw = level_dim(ti.w, ti.L); *sh = level_dim(ti.h, ti.L);
    return;
  }
  int64_t pw = level_dim(ti.w, level - 1), ph = level_dim(ti.h, level - 1);
  int64_t lw = (pw + 1) / 2, lh = (ph + 1) / 2;
  if (type == 0) { *x = lw; *y = 0; *sw = pw / 2; *sh = lh; }
  else if (type == 1) { *x = 0; *y = lh; *sw = lw; *sh = ph / 2; }
  else { *x = lw; *y = lh; *sw = pw / 2; *sh = ph / 2; }
}

int qlog2_of(const TileInfo& ti, int level) { return level == 0 ? ti.q[ti.L] : ti.q[level - 1]; }

// Gather block r from the Mallat planes into a padded Block.
Block gather_block(const TileInfo& ti, const std::vector<std::vector<int64_t>>& planes, const BlockRef& r) {
  Block b;
  b.p = r.level == 0 ? 1 : 3;
  int64_t gw = level_dim(ti.w, r.level == 0 ? ti.L : r.level);
  int64_t gh = level_dim(ti.h, r.level == 0 ? ti.L : r.level);
  int64_t bw = std::min<int64_t>(128, gw - 128 * r.bx), bh = std::min<int64_t>(128, gh - 128 * r.by);
  b.w = ceildiv(bw, 4) * 4; b.h = ceildiv(bh, 4) * 4;
  for (int t = 0; t < b.p; ++t) {
    int64_t x, y, sw, sh;
    subband_rect(ti, r.level, t, &x, &y, &sw, &sh);
    b.coef[t].assign((size_t)(b.w * b.h), 0);
    for (int64_t rr = 0; rr < b.h; ++rr)
      for (int64_t cc = 0; cc < b.w; ++cc) {
        int64_t sy = 128 * r.by + rr, sx = 128 * r.bx + cc;
        if (sy < sh && sx < sw) b.coef[t][rr * b.w + cc] = planes[r.c][(y + sy) * ti.w + (x + sx)];
      }
  }
  return b;
}

void scatter_block(const TileInfo& ti, std::vector<std::vector<int64_t>>& planes, const BlockRef& r, const Block& b) {
  for (int t = 0; t < b.p; ++t) {
    int64_t x, y, sw, sh;
    subband_rect(ti, r.level, t, &x, &y, &sw, &sh);
    for (int64_t rr = 0; rr < b.h; ++rr)
      for (int64_t cc = 0; cc < b.w; ++cc) {
        int64_t sy = 128 * r.by + rr, sx = 128 * r.bx + cc;
        if (sy < sh && sx < sw) planes[r.c][(y + sy) * ti.w + (x + sx)] = b.coef[t][rr * b.w + cc];
      }
  }
}

int64_t pixel_at(const void* px, int64_t pitch, int bits, int C, int64_t x, int64_t y, int c) {
  const uint8_t* row = (const uint8_t*)px + y * pitch;
  if (bits <= 8) return row[x * C + c];
  uint16_t v;
  std::memcpy(&v, row + 2 * (x * C + c), 2);
  return v;
}

void put_u16(uint8_t* p, uint32_t v) { p[0] = (uint8_t)v; p[1] = (uint8_t)(v >> 8); }
void put_u32(uint8_t* p, uint32_t v) { for (int i = 0; i < 4; ++i) p[i] = (uint8_t)(v >> (8 * i)); }
uint32_t get_u16(const uint8_t* p) { return (uint32_t)p[0] | ((uint32_t)p[1] << 8); }
uint32_t get_u32(const uint8_t* p) { uint32_t v = 0; for (int i = 0; i < 4; ++i) v |= (uint32_t)p[i] << (8 * i); return v; }

// Forward transform + quantisation of one tile into C Mallat planes.  The
// colour transform (Fig. 1, "optional") acts on channels 0..2; any further
// channels (and every channel of a tile without one) are coded as they are
// (Sec. 3: "an arbitrary number of channels").
std::vector<std::vector<int64_t>> tile_coefficients(const TileInfo& ti, const void* px, int64_t pitch) {
  std::vector<std::vector<int64_t>> planes(ti.C, std::vector<int64_t>((size_t)ti.w * ti.h));
  for (int64_t y = 0; y < ti.h; ++y)
    for (int64_t x = 0; x < ti.w; ++x) {
      for (int c = 0; c < ti.C; ++c) planes[c][y * ti.w + x] = pixel_at(px, pitch, ti.bits, ti.C, x, y, c);
      if (ti.ct != 0) {
        const int64_t R = planes[0][y * ti.w + x], G = planes[1][y * ti.w + x], B = planes[2][y * ti.w + x];
        int64_t a, b, c;
        if (ti.ct == 1) rct_forward(R, G, B, &a, &b, &c);
        else ycocg_forward(R, G, B, &a, &b, &c);
        planes[0][y * ti.w + x] = a; planes[1][y * ti.w + x] = b; planes[2][y * ti.w + x] = c;
      }
    }
  for (int c = 0; c < ti.C; ++c) {
    dwt2_forward(planes[c].data(), ti.w, ti.w, ti.h, ti.L);
    // quantise every subband with its own step
    for (int l = 0; l <= ti.L; ++l) {
      int types = l == 0 ? 1 : 3;
      for (int t = 0; t < types; ++t) {
        int64_t x0, y0, sw, sh;
        subband_rect(ti, l, t, &x0, &y0, &sw, &sh);
        int64_t delta = (int64_t)1 << qlog2_of(ti, l);
        for (int64_t y = 0; y < sh; ++y)
          for (int64_t x = 0; x < sw; ++x) {
            int64_t& v = planes[c][(y0 + y) * ti.w + x0 + x];
            v = quantise(v, delta);
          }
      }
    }
  }
  return planes;
}

bool tile_info_valid(const TileInfo& ti) {
  if (ti.w < 1 || ti.w > 65535 || ti.h < 1 || ti.h > 65535) return false;
  if (ti.C < 1 || ti.C > 16) return false;
  if (ti.ct < 0 || ti.ct > 2 || (ti.ct != 0 && ti.C < 3)) return false;
  if (ti.bits < 1 || ti.bits > 16) return false;
  if (ti.L < 0 || ti.L > 15) return false;
  for (int l = 0; l <= ti.L; ++l) if (ti.q[l] > 15) return false;
  return true;
}

std::vector<uint8_t> encode_tile(const TileInfo& ti, const void* px, int64_t pitch) {
  std::vector<std::vector<int64_t>> planes = tile_coefficients(ti, px, pitch);
  std::vector<BlockRef> refs = tile_blocks(ti);
  std::vector<uint8_t> data;
  std::vector<uint32_t> ends;
  for (const BlockRef& r : refs) {
    Block b = gather_block(ti, planes, r);
    std::vector<uint8_t> bytes = encode_block(b, nullptr);
    data.insert(data.end(), bytes.begin(), bytes.end());
    ends.push_back((uint32_t)data.size());
  }
  std::vector<uint8_t> out(32 + 4 * refs.size());
  out[0] = 'I'; out[1] = 'S'; out[2] = 'X'; out[3] = '1';
  put_u16(&out[4], (uint32_t)ti.w); put_u16(&out[6], (uint32_t)ti.h);
  out[8] = (uint8_t)ti.C; out[9] = (uint8_t)ti.bits; out[10] = (uint8_t)ti.L; out[11] = (uint8_t)ti.ct;
  put_u32(&out[12], (uint32_t)refs.size());
  for (int i = 0; i < 16; ++i) out[16 + i] = ti.q[i];
  for (size_t i = 0; i < ends.size(); ++i) put_u32(&out[32 + 4 * i], ends[i]);
  out.insert(out.end(), data.begin(), data.end());
  return out;
}

int parse_tile_header(const uint8_t* s, int64_t size, TileInfo& ti, uint32_t& nb) {
  if (size < 32 || s[0] != 'I' || s[1] != 'S' || s[2] != 'X' || s[3] != '1') return -1;
  ti.w = (int)get_u16(s + 4); ti.h = (int)get_u16(s + 6);
  ti.C = s[8]; ti.bits = s[9]; ti.L = s[10]; ti.ct = s[11];
  nb = get_u32(s + 12);
  for (int i = 0; i < 16; ++i) ti.q[i] = s[16 + i];
  if (!tile_info_valid(ti)) return -1;
  if ((int64_t)32 + 4 * (int64_t)nb > size) return -1;
  return 0;
}

// Decode a tile at resolution level z (Sec. 4: discard the high-pass blocks
// of the finer levels), dropping `drop` LSB planes.  Writes the
// ceil(w/2^z) x ceil(h/2^z) x C image (uint8 for bits <= 8, else uint16).
int decode_tile(const uint8_t* s, int64_t size, int z, int drop, void* out, int64_t pitch) {
  TileInfo ti;
  uint32_t nb;
  if (parse_tile_header(s, size, ti, nb) != 0) return -1;
  if (z < 0 || z > ti.L) return -1;
  std::vector<BlockRef> refs = tile_blocks(ti);
  if (refs.size() != nb) return -1;
  const uint8_t* data = s + 32 + 4 * (int64_t)nb;
  int64_t data_size = size - 32 - 4 * (int64_t)nb;
  std::vector<std::vector<int64_t>> planes(ti.C, std::vector<int64_t>((size_t)ti.w * ti.h, 0));
  uint32_t prev = 0;
  for (uint32_t i = 0; i < nb; ++i) {
    uint32_t end = get_u32(s + 32 + 4 * i);
    if (end < prev || (int64_t)end > data_size) return -1;
    const BlockRef& r = refs[i];
    if (r.level == 0 || r.level > z) {
      Block b;
      b.p = r.level == 0 ? 1 : 3;
      int64_t gw = level_dim(ti.w, r.level == 0 ? ti.L : r.level);
      int64_t gh = level_dim(ti.h, r.level == 0 ? ti.L : r.level);
      b.w = ceildiv(std::min<int64_t>(128, gw - 128 * r.bx), 4) * 4;
      b.h = ceildiv(std::min<int64_t>(128, gh - 128 * r.by), 4) * 4;
      if (decode_block(data + prev, end - prev, b, drop) != 0) return -1;
      scatter_block(ti, planes, r, b);
    }
    prev = end;
  }
  int64_t zw = level_dim(ti.w, z), zh = level_dim(ti.h, z);
  for (int c = 0; c < ti.C; ++c) {
    for (int l = 0; l <= ti.L; ++l) {
      if (l != 0 && l <= z) continue;
      int types = l == 0 ? 1 : 3;
      for (int t = 0; t < types; ++t) {
        int64_t x0, y0, sw, sh;
        subband_rect(ti, l, t, &x0, &y0, &sw, &sh);
        int64_t delta = (int64_t)1 << qlog2_of(ti, l);
        for (int64_t y = 0; y < sh; ++y)
          for (int64_t x = 0; x < sw; ++x) {
            int64_t& v = planes[c][(y0 + y) * ti.w + x0 + x];
            v = dequantise(v, delta);
          }
      }
    }
    dwt2_inverse(planes[c].data(), ti.w, zw, zh, ti.L - z);
  }
  int64_t maxv = ((int64_t)1 << ti.bits) - 1;
  for (int64_t y = 0; y < zh; ++y)
    for (int64_t x = 0; x < zw; ++x) {
      int64_t v[16];
      for (int c = 0; c < ti.C; ++c) v[c] = planes[c][y * ti.w + x];
      if (ti.ct == 1) rct_inverse(v[0], v[1], v[2], &v[0], &v[1], &v[2]);
      else if (ti.ct == 2) ycocg_inverse(v[0], v[1], v[2], &v[0], &v[1], &v[2]);
      for (int c = 0; c < ti.C; ++c) {
        int64_t q = std::min(std::max(v[c], (int64_t)0), maxv);
        uint8_t* row = (uint8_t*)out + y * pitch;
        if (ti.bits <= 8) row[x * ti.C + c] = (uint8_t)q;
        else { uint16_t u = (uint16_t)q; std::memcpy(row + 2 * (x * ti.C + c), &u, 2); }
      }
    }
  return 0;
}

}  // namespace

// =================================================================== C ABI
// Used through ctypes by the tests and the benchmark's CPU-baseline leg.
extern "C" {

// transform: 0 = RCT for three channels and none otherwise, 1 = none,
// 2 = RCT, 3 = YCoCg-R (2 and 3 on channels 0..2 of a tile of 3 or more).
typedef struct {
  int32_t width, height, channels, bits, levels, x0, y0;
  uint8_t qstep_log2[16];
  int32_t transform;
} orc_tile;

static TileInfo to_info(const orc_tile* t) {
  TileInfo ti;
  ti.w = t->width; ti.h = t->height; ti.C = t->channels; ti.bits = t->bits; ti.L = t->levels;
  ti.ct = t->transform == 0 ? (t->channels == 3 ? 1 : 0) : t->transform == 1 ? 0 : t->transform == 2 ? 1 : t->transform == 3 ? 2 : -1;
  for (int i = 0; i < 16; ++i) ti.q[i] = i <= t->levels ? t->qstep_log2[i] : 0;
  return ti;
}

// --- step-level entry points (pins) ---
void orc_rct_forward(const int64_t* rgb, int64_t n, int64_t* ycc) {
  for (int64_t i = 0; i < n; ++i) rct_forward(rgb[3 * i], rgb[3 * i + 1], rgb[3 * i + 2], &ycc[3 * i], &ycc[3 * i + 1], &ycc[3 * i + 2]);
}
void orc_rct_inverse(const int64_t* ycc, int64_t n, int64_t* rgb) {
  for (int64_t i = 0; i < n; ++i) rct_inverse(ycc[3 * i], ycc[3 * i + 1], ycc[3 * i + 2], &rgb[3 * i], &rgb[3 * i + 1], &rgb[3 * i + 2]);
}
void orc_ycocg_forward(const int64_t* rgb, int64_t n, int64_t* ycc) {
  for (int64_t i = 0; i < n; ++i) ycocg_forward(rgb[3 * i], rgb[3 * i + 1], rgb[3 * i + 2], &ycc[3 * i], &ycc[3 * i + 1], &ycc[3 * i + 2]);
}
void orc_ycocg_inverse(const int64_t* ycc, int64_t n, int64_t* rgb) {
  for (int64_t i = 0; i < n; ++i) ycocg_inverse(ycc[3 * i], ycc[3 * i + 1], ycc[3 * i + 2], &rgb[3 * i], &rgb[3 * i + 1], &rgb[3 * i + 2]);
}
void orc_lift53_forward(const int64_t* x, int64_t n, int64_t* low, int64_t* high) { lift53_forward(x, n, low, high); }
void orc_lift53_inverse(const int64_t* low, const int64_t* high, int64_t n, int64_t* x) { lift53_inverse(low, high, n, x); }
void orc_dwt2_forward(int64_t* plane, int64_t w, int64_t h, int levels) { dwt2_forward(plane, w, w, h, levels); }
void orc_dwt2_inverse(int64_t* plane, int64_t w, int64_t h, int levels) { dwt2_inverse(plane, w, w, h, levels); }
int64_t orc_quantise(int64_t c, int64_t delta) { return quantise(c, delta); }
int64_t orc_dequantise(int64_t q, int64_t delta) { return dequantise(q, delta); }
void orc_area_T(int64_t k, int64_t w, int64_t h, int64_t* ijp) { area_T(k, w, h, &ijp[0], &ijp[1], &ijp[2]); }
int orc_area_symbol(const int64_t* coef, int64_t w, int64_t i, int64_t j, int64_t p, int64_t d) { return area_symbol(coef, w, i, j, p, d); }

// Huffman: freq[256] -> len[256] (-1 absent), code[256]; tree bits into
// tree_out (returns number of tree bits).
int64_t orc_huffman(const uint64_t* freq, int32_t* len, uint32_t* code, uint8_t* tree_out, int64_t tree_cap) {
  HuffCode hc = huffman_build(freq);
  for (int s = 0; s < 256; ++s) { len[s] = hc.len[s]; code[s] = hc.code[s]; }
  if (hc.n_leaves == 0) return 0;
  BitWriter bw;
  huffman_write_tree(hc, hc.root, bw);
  for (size_t i = 0; i < bw.bytes.size() && (int64_t)i < tree_cap; ++i) tree_out[i] = bw.bytes[i];
  return (int64_t)bw.nbits;
}

// Zero-run tokenisation of one segment: writes (symbol, run) pairs.
int64_t orc_tokens(const int32_t* seg, int64_t n, int czr, int w, int32_t* sym_out, int64_t* run_out, int64_t cap) {
  std::vector<int> s(seg, seg + n);
  std::vector<Token> t = tokens_of(find_runs(s), czr, w);
  for (size_t i = 0; i < t.size() && (int64_t)i < cap; ++i) { sym_out[i] = t[i].symbol; run_out[i] = t[i].run; }
  return (int64_t)t.size();
}

// Block codec on explicit coefficients: coef = p planes of h x w (padded).
// stats_out (8 + 256 int64): d, czr, w, t, b, l_prov, n_sym, 0, then the
// provisional code's length of each symbol 0..255 (0 = absent).
int64_t orc_encode_block(int p, int64_t w, int64_t h, const int64_t* coef, uint8_t* out, int64_t cap, int64_t* stats_out) {
  Block b;
  b.p = p; b.w = w; b.h = h;
  for (int t = 0; t < p; ++t) b.coef[t].assign(coef + t * w * h, coef + (t + 1) * w * h);
  EncodeStats st;
  std::vector<uint8_t> bytes = encode_block(b, &st);
  if (stats_out) {
    stats_out[0] = st.d; stats_out[1] = st.czr; stats_out[2] = st.w; stats_out[3] = st.t;
    stats_out[4] = st.b; stats_out[5] = st.l_prov; stats_out[6] = st.n_sym; stats_out[7] = 0;
    for (int s = 0; s < 256; ++s) stats_out[8 + s] = st.prov_len[s];
  }
  if ((int64_t)bytes.size() > cap) return -(int64_t)bytes.size();
  std::memcpy(out, bytes.data(), bytes.size());
  return (int64_t)bytes.size();
}

int orc_decode_block(int p, int64_t w, int64_t h, const uint8_t* data, int64_t size, int drop, int64_t* coef) {
  Block b;
  b.p = p; b.w = w; b.h = h;
  int rc = decode_block(data, size, b, drop);
  if (rc != 0) return rc;
  for (int t = 0; t < p; ++t) std::memcpy(coef + t * w * h, b.coef[t].data(), (size_t)(w * h) * sizeof(int64_t));
  return 0;
}

// Coefficients of a whole tile (after colour transform, wavelet and
// quantisation), C Mallat planes of w x h.
int orc_tile_coefficients(const orc_tile* t, const void* px, int64_t pitch, int64_t* out) {
  TileInfo ti = to_info(t);
  if (!tile_info_valid(ti)) return -1;
  std::vector<std::vector<int64_t>> planes = tile_coefficients(ti, px, pitch);
  for (int c = 0; c < ti.C; ++c) std::memcpy(out + (int64_t)c * ti.w * ti.h, planes[c].data(), (size_t)ti.w * ti.h * sizeof(int64_t));
  return 0;
}

// --- tile codec ---
// Returns the stream size; a negative value -n means the capacity was too
// small and n bytes are needed; 0 means invalid arguments.
int64_t orc_encode_tile(const orc_tile* t, const void* px, int64_t pitch, uint8_t* out, int64_t cap) {
  TileInfo ti = to_info(t);
  if (!tile_info_valid(ti)) return 0;
  std::vector<uint8_t> s = encode_tile(ti, px, pitch);
  if ((int64_t)s.size() > cap) return -(int64_t)s.size();
  std::memcpy(out, s.data(), s.size());
  return (int64_t)s.size();
}

int orc_decode_tile(const uint8_t* s, int64_t size, int level, int drop, void* out, int64_t pitch) {
  return decode_tile(s, size, level, drop, out, pitch);
}

// Many tiles at once on a pool of std::threads, one tile per task (the
// CPU baseline).  Each tile i reads px[i] with pitch[i] and writes to
// out[i] (capacity cap[i]); sizes[i] receives orc_encode_tile's result.
void orc_encode_tiles_mt(int64_t n, const orc_tile* tiles, const void* const* px, const int64_t* pitch,
                         uint8_t* const* out, const int64_t* cap, int64_t* sizes, int threads) {
  std::atomic<int64_t> next(0);
  auto work = [&]() {
    for (;;) {
      int64_t i = next.fetch_add(1);
      if (i >= n) break;
      sizes[i] = orc_encode_tile(&tiles[i], px[i], pitch[i], out[i], cap[i]);
    }
  };
  if (threads < 1) threads = 1;
  std::vector<std::thread> pool;
  for (int k = 0; k < threads; ++k) pool.emplace_back(work);
  for (auto& th : pool) th.join();
}

void orc_decode_tiles_mt(int64_t n, const uint8_t* const* s, const int64_t* size, int level,
                         void* const* out, const int64_t* pitch, int32_t* rc, int threads) {
  std::atomic<int64_t> next(0);
  auto work = [&]() {
    for (;;) {
      int64_t i = next.fetch_add(1);
      if (i >= n) break;
      rc[i] = decode_tile(s[i], size[i], level, 0, out[i], pitch[i]);
    }
  };
  if (threads < 1) threads = 1;
  std::vector<std::thread> pool;
  for (int k = 0; k < threads; ++k) pool.emplace_back(work);
  for (auto& th : pool) th.join();
}

}  // extern "C"
