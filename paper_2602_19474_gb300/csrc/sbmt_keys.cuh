// sbmt_keys.cuh -- the registry of the template retriangulation (App. G):
// the key codes of the finite lookup table in its canonical frame and, per
// (key, rotation), the patch's triangles in local labels; and the (m, n)
// class index of Thm. 3.2.  Shared by the lattice path (k_cells.cu) and the
// retriangulation of the preprocessed mesh (k_region3.cu), so that both
// look up the same single-valued table (Assumption "frozen registry and
// single-valued lookup").
#pragma once
#include "sbmt_dev.cuh"

namespace sbmt {

namespace {

// ---------------------------------------------------------------------------
// lookup table (App. G), canonical frame: labels 0,1,2 = A', B', C';
// 3..6 = E0..E3, the events read counter-clockwise from A'; 7 = P
// ---------------------------------------------------------------------------
enum { TA = 0, TB = 1, TC = 2, T0 = 3, T1 = 4, T2 = 5, T3 = 6, TP = 7 };
constexpr int NKEYS = 15;
// canonical code star<<10 | n(A'B')<<7 | n(B'C')<<4 | n(C'A')<<1 | dir of keys 1..15
constexpr unsigned short kKeyCode[NKEYS] = {
    (0 << 10) | (0 << 7) | (1 << 4) | (1 << 1) | 0,  // 1 single segment (b)
    (1 << 10) | (0 << 7) | (1 << 4) | (1 << 1) | 0,  // 2 (1,1) (a)
    (1 << 10) | (0 << 7) | (0 << 4) | (2 << 1) | 0,  // 3 (1,1) (c)
    (0 << 10) | (1 << 7) | (1 << 4) | (2 << 1) | 0,  // 4 (2,2) (b1)
    (0 << 10) | (0 << 7) | (2 << 4) | (2 << 1) | 1,  // 5 (2,2) (d3)
    (0 << 10) | (0 << 7) | (2 << 4) | (2 << 1) | 0,  // 6 (2,2) (a4)
    (1 << 10) | (0 << 7) | (0 << 4) | (3 << 1),      // 7..15: one vertex of degree 3-4,
    (1 << 10) | (0 << 7) | (1 << 4) | (2 << 1),      //   star from P
    (1 << 10) | (0 << 7) | (2 << 4) | (1 << 1),
    (1 << 10) | (1 << 7) | (1 << 4) | (1 << 1),
    (1 << 10) | (0 << 7) | (0 << 4) | (4 << 1),
    (1 << 10) | (0 << 7) | (1 << 4) | (3 << 1),
    (1 << 10) | (0 << 7) | (2 << 4) | (2 << 1),
    (1 << 10) | (0 << 7) | (3 << 4) | (1 << 1),
    (1 << 10) | (1 << 7) | (1 << 4) | (2 << 1),
};
// templates of the paper's keys 1..6, in App. G's order
constexpr unsigned char kTpl[6][5][3] = {
    // single segment (b): Q1 on B'C' (E0), Q2 on C'A' (E1)
    {{T1, T0, TC}, {T1, TA, TB}, {T0, T1, TB}, {0, 0, 0}, {0, 0, 0}},
    // (1,1) (a): Q2 on B'C' (E0), Q1 on C'A' (E1), P inside
    {{T1, TP, TC}, {TP, T0, TC}, {T1, TA, TP}, {TA, TB, TP}, {T0, TP, TB}},
    // (1,1) (c): Q1, Q2 on C'A', Q1 nearer C' (E0 = Q1, E1 = Q2)
    {{T0, TP, TC}, {TP, T0, T1}, {T1, TA, TP}, {TB, TC, TP}, {TA, TB, TP}},
    // (2,2) (b1): Q1 on A'B' (E0), Q3 on B'C' (E1), Q4 (E2) and Q2 (E3) on C'A'
    {{T0, T3, TA}, {T0, T2, T3}, {T0, T1, T2}, {T0, TB, T1}, {T2, T1, TC}},
    // (2,2) (d3): nested chords at C'; Q4 (E0), Q3 (E1) on B'C'; Q1 (E2), Q2 (E3) on C'A'
    {{TA, TB, T3}, {T3, TB, T0}, {T2, T3, T0}, {T2, T0, T1}, {T2, T1, TC}},
    // (2,2) (a4), drawn at A and turned so the cut corner is C': Q2 (E0), Q1 (E1)
    // on B'C'; Q3 (E2), Q4 (E3) on C'A'
    {{T2, T1, TC}, {T3, T1, T2}, {T1, T3, T0}, {T0, T3, TA}, {T0, TA, TB}},
};

// The registry as the kernels read it: the key codes, and per (key, sigma)
// the patch's triangles in local labels (0..2 the corners A, B, C; 3.. the
// events in counter-clockwise order from A; 7 the inside vertex P), three
// 3-bit labels per triangle, triangle k in bits 9k..9k+8.  The template is
// read through sigma (Alg. 2 "instantiate by a single map"): canonical
// corner k is corner (sigma + k) mod 3, canonical edge s is edge
// (sigma + s) mod 3, and the key's code holds the event count of each
// canonical edge.
struct KeyTable {
  unsigned short code[NKEYS];
  unsigned long long tris[NKEYS * 3];
};
constexpr KeyTable make_key_table() {
  KeyTable t{};
  for (int k = 0; k < NKEYS; ++k) t.code[k] = kKeyCode[k];
  for (int key = 1; key <= NKEYS; ++key)
    for (int sigma = 0; sigma < 3; ++sigma) {
      const unsigned kc = kKeyCode[key - 1];
      const int ncan[3] = {(int)((kc >> 7) & 7u), (int)((kc >> 4) & 7u), (int)((kc >> 1) & 7u)};
      int nin[3] = {0, 0, 0};
      for (int s = 0; s < 3; ++s) nin[(sigma + s) % 3] = ncan[s];
      int map[8] = {0, 0, 0, 0, 0, 0, 0, 7};
      for (int k = 0; k < 3; ++k) map[k] = (sigma + k) % 3;
      int tt = 0;
      for (int s = 0; s < 3; ++s) {
        const int e = (sigma + s) % 3;
        int first = 3;
        for (int u = 0; u < e; ++u) first += nin[u];
        for (int u = 0; u < nin[e]; ++u) map[3 + tt++] = first + u;
      }
      unsigned long long w = 0;
      auto put = [&](int k, int a, int b, int c) {
        w |= (unsigned long long)(map[a] | map[b] << 3 | map[c] << 6) << (9 * k);
      };
      if (key <= 6) {
        const int nt = key == 1 ? 3 : 5;
        for (int k = 0; k < nt; ++k) put(k, kTpl[key - 1][k][0], kTpl[key - 1][k][1], kTpl[key - 1][k][2]);
      } else {
        // star from P over the boundary cycle read counter-clockwise from A'
        int cyc[8] = {}, nc = 0, ev_i = 0;
        for (int s = 0; s < 3; ++s) {
          cyc[nc++] = s;
          for (int u = 0; u < ncan[s]; ++u) cyc[nc++] = T0 + ev_i++;
        }
        for (int k = 0; k < nc; ++k) put(k, cyc[k], cyc[(k + 1) % nc], TP);
      }
      t.tris[(key - 1) * 3 + sigma] = w;
    }
  return t;
}
__device__ const KeyTable g_keys = make_key_table();

// local labels of triangle k of a packed patch
SBMT_DEV int tri_label(unsigned long long w, int k, int u) { return (int)((w >> (9 * k + 3 * u)) & 7u); }

SBMT_DEV int thm32_class(int m, int n) {
  // 1-based position of the sorted pair in Thm. 3.2's list, 0 if absent
  const int lo = m < n ? m : n, hi = m < n ? n : m;
  switch (lo * 4 + hi) {
    case 0 * 4 + 1: return 1;
    case 0 * 4 + 2: return 2;
    case 0 * 4 + 3: return 3;
    case 1 * 4 + 1: return 4;
    case 1 * 4 + 2: return 5;
    case 2 * 4 + 2: return 6;
    case 1 * 4 + 3: return 7;
    case 2 * 4 + 3: return 8;
    default: return 0;
  }
}

}  // namespace

}  // namespace sbmt
