// Host-side choice of the fold's work split and of its epilogue tables: plain C++ with no
// CUDA calls, used by the plan (capi.cu) and compiled on its own by the host tests.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <utility>
#include <vector>

#include "device.cuh"

namespace rsft {

inline int ceil_log2(int64_t v) {
  int r = 0;
  while ((int64_t(1) << r) < v) ++r;
  return r;
}

// Choose how the fold splits rows and columns (see fold.cu).  Costs are relative to
// the 8 bytes each cube element costs: per-element row-weight setup and partial-sum traffic.
// Scores every fold schedule the kernels support and returns the cheapest; with `all`, also
// every candidate with its model cost (the autotuner times the best few).
inline bool choose_fold_schedule(const Geometry& g, int sms, FoldSchedule& out,
                                 std::vector<std::pair<double, FoldSchedule>>* all = nullptr,
                                 int group = kMaxLoopGroup) {
  const int lg = std::min(g.loops, group);
  double best = 1e300;
  bool found = false;
  for (int d_in = 0; d_in < g.ndim; ++d_in) {
    int64_t row_len = 1, rows_pc = 1, classes = 1, xcount = 1, after = 1;
    for (int e = d_in; e < g.ndim; ++e) {
      row_len *= g.n[e];
      xcount *= g.b[e];
    }
    for (int e = d_in + 1; e < g.ndim; ++e) after *= g.n[e];
    for (int e = 0; e < d_in; ++e) {
      rows_pc *= g.m[e];
      classes *= g.b[e];
    }
    const int64_t width = std::min<int64_t>(row_len, 2 * kFoldConsumers);
    if (width < row_len) {
      // a chunk must hold whole residue periods: W = w_p * prod_{e > d_in} N_e, B_{d_in} | w_p
      if (width % after != 0) continue;
      if ((width / after) % g.b[d_in] != 0) continue;
    }
    if (xcount > width || xcount > 65535) continue;
    if (classes > (int64_t(1) << 30)) continue;
    // C classes side by side in a step: consecutive residues of the innermost row dimension
    int64_t cmax = 1;
    if (d_in >= 1)
      while (cmax * 2 * width <= 2 * kFoldConsumers && cmax * 2 <= g.b[d_in - 1] && cmax * 2 <= classes) cmax *= 2;
    for (int64_t cps = 1; cps <= cmax; cps *= 2) {
      const int64_t rpc = rows_pc;  // whole classes per unit (direct output unless columns are chunked)
      const int64_t crow = std::min<int64_t>(2 * kFoldConsumers / (width * cps), rpc);
      const int64_t row_chunks = 1;
      const int64_t col_chunks = row_len / width;
      const int64_t units = classes / cps * row_chunks * col_chunks;
      if (units > 0x7fffffff || rpc > (int64_t(1) << 30)) continue;
      const double setup = static_cast<double>(lg) / static_cast<double>(width * cps * crow / 2);
      const double partial = (row_chunks * col_chunks > 1)
                                 ? 2.0 * lg * static_cast<double>(xcount) / static_cast<double>(rpc * width)
                                 : 0.0;
      const double idle = 1.0 - static_cast<double>(width * cps * crow) / (2 * kFoldConsumers);
      // persistent CTAs (two per SM) take units round robin and each runs at about a fixed
      // rate: the busiest CTA's units against an even share, plus a per-unit cost (epilogue,
      // ring refill) worth about 3072 elements of the row loop
      const double slots = 2.0 * sms;
      const double per_cta = std::ceil(static_cast<double>(units) / slots);
      const double balance = std::min(4.0, per_cta / (static_cast<double>(units) / slots) - 1.0) +
                             3072.0 / static_cast<double>(cps * rpc * width);
      // rows without a tensor map go as one bulk copy each: small ones are request-rate bound
      const bool tensor_map = d_in >= 1 && d_in <= 2 && width <= 256;
      const double copies = (!tensor_map && width < 256) ? 1.0 : 0.0;
      const double cost = 0.5 * setup + partial + balance + idle + copies;
      FoldSchedule c{};
      c.d_in = d_in;
      c.row_len = row_len;
      c.width = static_cast<int>(width);
      c.col_chunks = static_cast<int>(col_chunks);
      c.classes = static_cast<int>(classes);
      c.rows_per_class = static_cast<int>(rows_pc);
      c.rows_per_chunk = static_cast<int>(rpc);
      c.row_chunks = static_cast<int>(row_chunks);
      c.xcount = static_cast<int>(xcount);
      c.direct = (row_chunks * col_chunks == 1) ? 1 : 0;
      c.cps = static_cast<int>(cps);
      c.crow = static_cast<int>(crow);
      c.groups = static_cast<int>(classes / cps);
      if (all) all->emplace_back(cost, c);
      if (cost < best - 1e-9) {
        best = cost;
        found = true;
        out = c;
      }
    }
  }
  return found;
}


// Inner residue index of chunk column c: the residues s_d mod B_d of the column dimensions
// [d_in, D), mixed-radix with the last dimension fastest.
inline int64_t fold_residue(const int64_t* n, const int64_t* b, int D, const FoldSchedule& fs, int64_t c) {
  int64_t rem = c, x = 0, xstride = 1;
  for (int d = D - 1; d >= fs.d_in; --d) {
    const int64_t sd = rem % n[d];
    rem /= n[d];
    x += (sd % b[d]) * xstride;
    xstride *= b[d];
  }
  return x;
}

// The epilogue of a chosen schedule: which column pair each thread holds (fs.lane_perm), the
// lane bits the warp shuffle sums (fs.red_mask, fs.leaders), and per (class in step, inner
// residue) the list of partial sums left after the shuffle (slots, fs.slots_per_x entries
// each), plus the residue digits of each inner residue ([X][4]).  Returns nullptr, or the
// reason the schedule cannot be used.
inline const char* fold_epilogue_tables(const int64_t* n, const int64_t* b, int D, FoldSchedule& fs,
                                        std::vector<unsigned short>& slots, std::vector<unsigned short>& digits) {
  // element bit e of a row step: a column bit or, past the chunk width, a row bit (the class
  // of the row for the first log2 C row bits, then its row); does flipping it keep the
  // thread's (class, inner residue)?
  auto keeps = [&](int e) {
    if ((int64_t(1) << e) >= fs.width) return ((int64_t(1) << e) / fs.width) >= fs.cps;
    int acc = 0;
    for (int d = D - 1; d >= fs.d_in; --d) {
      const int ln = ceil_log2(n[d]);
      if (e < acc + ln) return (e - acc) >= ceil_log2(b[d]);
      acc += ln;
    }
    return true;
  };
  // thread -> column pair: thread bits 0-2 stay on pair bits 0-2 (a quarter warp reads 128
  // contiguous bytes, free of bank conflicts); when a chunk row has more than 32 pairs,
  // thread bits 3-4 take the lowest pair bits that keep the residue, so the warp shuffle
  // sums them instead of the epilogue's shared-memory partials
  int perm[8] = {0, 1, 2, 3, 4, 5, 6, 7};
  const int pair_bits = ceil_log2(fs.width / 2);
  if (pair_bits > 5) {
    std::vector<int> first, rest;
    for (int pb = 3; pb < pair_bits; ++pb) (keeps(pb + 1) && first.size() < 2 ? first : rest).push_back(pb);
    first.insert(first.end(), rest.begin(), rest.end());
    for (int q = 3; q < pair_bits; ++q) perm[q] = first[q - 3];
  }
  fs.lane_perm = 0;
  for (int q = 0; q < 8; ++q) fs.lane_perm |= static_cast<unsigned>(perm[q]) << (4 * q);
  // lane bit k moves a thread's pair index by 2^perm[k], its elements by twice that
  int rmask = 0;
  for (int k = 0; k < 5; ++k)
    if (keeps(perm[k] + 1)) rmask |= 1 << k;
  int nbits = 0;
  for (int k = 0; k < 5; ++k) nbits += (rmask >> k) & 1;
  fs.red_mask = rmask;
  fs.leaders = 32 >> nbits;
  const int warps = kFoldConsumers / 32;
  const int nslots = warps * fs.leaders * 2;
  const int keys = fs.cps * fs.xcount;  // (class in step, inner residue)
  if (nslots % keys != 0) return "fold epilogue: residues not balanced";
  fs.slots_per_x = nslots / keys;
  if (nslots > 512 || fs.xcount > 512) return "fold epilogue: too many residues";
  slots.assign(static_cast<size_t>(nslots), 0);
  digits.assign(static_cast<size_t>(fs.xcount) * 4, 0);
  std::vector<int> fill(keys, 0);
  for (int w = 0; w < warps; ++w)
    for (int j = 0; j < fs.leaders; ++j) {
      int lane = 0, bit = 0;
      for (int q = 0; q < 5; ++q)
        if (!((rmask >> q) & 1)) lane |= ((j >> bit++) & 1) << q;
      for (int c = 0; c < 2; ++c) {
        const int64_t elem = 2 * static_cast<int64_t>(fold_pair_of(32 * w + lane, fs.lane_perm)) + c;
        const int64_t x = ((elem / fs.width) % fs.cps) * fs.xcount + fold_residue(n, b, D, fs, elem & (fs.width - 1));
        if (fill[x] >= fs.slots_per_x) return "fold epilogue: residues not balanced";
        slots[x * fs.slots_per_x + fill[x]++] = static_cast<unsigned short>((w * fs.leaders + j) * 2 + c);
      }
    }
  for (int x = 0; x < fs.xcount; ++x) {
    int64_t rem = x;
    for (int d = D - 1; d >= fs.d_in; --d) {
      digits[x * 4 + (d - fs.d_in)] = static_cast<unsigned short>(rem % b[d]);
      rem /= b[d];
    }
  }
  return nullptr;
}

}  // namespace rsft
