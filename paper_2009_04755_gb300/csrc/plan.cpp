// plan.cpp -- host-side schedule of the all-pairs library.
//
// The upper triangle of the item grid is walked in recursively blocked tiles
// (Sec. IV-B: the matrix is split into four quadrants, each quadrant again,
// quadrants without work are skipped).  Here the recursion stops at blocks of
// items; the resulting list of block pairs (I <= J) is what the persistent
// kernels pop from their atomic queue, so consecutive tiles share item blocks
// and stay warm in L2 and shared memory.
#include <algorithm>
#include <cstdint>
#include <vector>

#include "ap_internal.h"

namespace ap {

namespace {
struct Region { int64_t r0, r1, c0, c1; };
}

void dc_block_pairs(int64_t nb, std::vector<int32_t> &out) {
  out.clear();
  if (nb <= 0) return;
  // explicit stack; children pushed in reverse so they pop as TL, TR, BL, BR
  std::vector<Region> stack;
  stack.push_back({0, nb, 0, nb});
  while (!stack.empty()) {
    Region g = stack.back();
    stack.pop_back();
    if (g.r0 >= g.r1 || g.c0 >= g.c1) continue;
    if (g.r0 > g.c1 - 1) continue;            // every block below the diagonal
    if (g.r1 - g.r0 == 1 && g.c1 - g.c0 == 1) {
      out.push_back((int32_t)g.r0);           // block pair (I, J), I <= J
      out.push_back((int32_t)g.c0);
      continue;
    }
    int64_t rm = g.r0 + (g.r1 - g.r0 + 1) / 2;
    int64_t cm = g.c0 + (g.c1 - g.c0 + 1) / 2;
    stack.push_back({rm, g.r1, cm, g.c1});    // bottom-right (visited last)
    stack.push_back({rm, g.r1, g.c0, cm});    // bottom-left
    stack.push_back({g.r0, rm, cm, g.c1});    // top-right
    stack.push_back({g.r0, rm, g.c0, cm});    // top-left (visited first)
  }
}

void make_blocks(const std::vector<int64_t> &poff, const std::vector<int64_t> &cnt,
                 int32_t max_items, int64_t max_pts, int64_t chunk, int64_t max_chunks,
                 std::vector<int32_t> &bstart) {
  bstart.clear();
  int64_t n = (int64_t)poff.size() - 1;
  int64_t i = 0;
  while (i < n) {
    bstart.push_back((int32_t)i);
    int64_t pts = 0, k = 0, ch = 0;
    while (i < n && k < max_items) {
      int64_t sz = poff[i + 1] - poff[i];
      int64_t c = (cnt[i] + chunk - 1) / chunk;
      if (k > 0 && (pts + sz > max_pts || ch + c > max_chunks)) break;
      pts += sz;
      ch += c;
      ++k;
      ++i;
    }
  }
  bstart.push_back((int32_t)n);
}

int32_t max_row_jobs(const std::vector<int32_t> &bstart, const std::vector<int64_t> &cnt,
                     int64_t chunk) {
  int64_t best = 1;
  for (size_t b = 0; b + 1 < bstart.size(); ++b) {
    int64_t jobs = 0;
    for (int32_t i = bstart[b]; i < bstart[b + 1]; ++i) jobs += (cnt[i] + chunk - 1) / chunk;
    best = std::max(best, jobs);
  }
  return (int32_t)std::min<int64_t>(best, kOverlapMaxRowJobs);
}

void tc_tiles(int64_t n, std::vector<int32_t> &tiles) {
  // macro grid of kTcTileN items; each macro pair (I <= J) holds two row
  // halves of kTcTileM items, kept when they contain some pair i < j.
  tiles.clear();
  int64_t nb = (n + kTcTileN - 1) / kTcTileN;
  std::vector<int32_t> macro;
  dc_block_pairs(nb, macro);
  const int64_t halves = kTcTileN / kTcTileM;
  for (size_t t = 0; t < macro.size(); t += 2) {
    int64_t I = macro[t], J = macro[t + 1];
    for (int64_t h = 0; h < halves; ++h) {
      int64_t ib = I * halves + h;
      int64_t i0 = ib * kTcTileM;
      int64_t jmax = std::min<int64_t>(J * kTcTileN + kTcTileN, n) - 1;
      if (i0 >= n || i0 >= jmax) continue;   // no i < j in this half
      tiles.push_back((int32_t)ib);
      tiles.push_back((int32_t)J);
    }
  }
}

void panel_units(const std::vector<int32_t> &tiles, int64_t nchunks, int64_t group,
                 int64_t k_split, std::vector<int32_t> &units) {
  // waves of `group` consecutive tiles; inside a wave, column range p of
  // every tile before range p + 1 of any, so the tiles running at one time
  // stream the same columns of their rows
  units.clear();
  const int64_t nt = (int64_t)tiles.size() / 2;
  k_split = std::max<int64_t>(1, std::min<int64_t>(k_split, nchunks));
  for (int64_t w0 = 0; w0 < nt; w0 += group) {
    const int64_t w1 = std::min<int64_t>(nt, w0 + group);
    for (int64_t p = 0; p < k_split; ++p) {
      const int32_t c0 = (int32_t)(p * nchunks / k_split);
      const int32_t c1 = (int32_t)((p + 1) * nchunks / k_split);
      for (int64_t t = w0; t < w1; ++t) {
        const int32_t ib = tiles[2 * t], jb = tiles[2 * t + 1];
        const int32_t rb = jb * (kTcTileN / kTcTileM);
        const int32_t u[kOocTileInts] = {ib, rb, rb + 1, ib, jb, c0, c1, 0};
        units.insert(units.end(), u, u + kOocTileInts);
      }
    }
  }
}

void pair_units(int64_t n, int64_t nchunks, int64_t group, int64_t k_split,
                std::vector<int32_t> &units) {
  std::vector<int32_t> macro;
  dc_block_pairs((n + kTcTileN - 1) / kTcTileN, macro);
  pair_units_of(macro, nchunks, group, k_split, units);
}

void pair_units_of(const std::vector<int32_t> &macro, int64_t nchunks, int64_t group,
                   int64_t k_split, std::vector<int32_t> &units) {
  // macro pairs of 256 items; each CTA of a pair takes one 128-item half of
  // the I macro and stages one half of the J macro
  units.clear();
  const int64_t nt = (int64_t)macro.size() / 2;
  k_split = std::max<int64_t>(1, std::min<int64_t>(k_split, nchunks));
  group = std::max<int64_t>(1, group);
  for (int64_t w0 = 0; w0 < nt; w0 += group) {
    const int64_t w1 = std::min<int64_t>(nt, w0 + group);
    for (int64_t p = 0; p < k_split; ++p) {
      const int32_t c0 = (int32_t)(p * nchunks / k_split);
      const int32_t c1 = (int32_t)((p + 1) * nchunks / k_split);
      for (int64_t t = w0; t < w1; ++t) {
        const int32_t I = macro[2 * t], J = macro[2 * t + 1];
        const int32_t u[kOocTileInts] = {2 * I, 2 * I + 1, 2 * J, 2 * J + 1, 2 * I, J, c0, c1};
        units.insert(units.end(), u, u + kOocTileInts);
      }
    }
  }
}

}  // namespace ap
