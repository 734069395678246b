// Host-side check of the persistent work split shared by the tensor-core kernels
// (tc_common.cuh), run on the CPU: for many (row blocks R, column tiles T, CTAs G) every
// (row block, tile) unit is covered by exactly one segment; the CTAs whose segments touch
// a row block are exactly contributors() in CTA order, with seg_of() giving each one's
// segment index; the whole row blocks of the bands go to one CTA each. Exit status 0 on
// success, 1 with a message on the first violation.
#include <cstdint>
#include <cstdio>
#include <vector>

#include "../../paper_2406_05061_gb300/csrc/tc_common.cuh"

using progot::tc::Seg;
using progot::tc::Split;

static int check(int R, int T, int sms) {
  const int64_t units = (int64_t)R * T;
  const int G = (int)(units < sms ? units : sms);
  const Split s = progot::tc::make_split(R, T, G);
  std::vector<int> cover((size_t)units, -1);
  std::vector<std::vector<std::pair<int, int>>> touch((size_t)R);
  for (int c = 0; c < G; ++c) {
    const int ns = progot::tc::num_segments(s, c);
    for (int k = 0; k < ns; ++k) {
      const Seg sg = progot::tc::segment(s, c, k);
      if (sg.r < 0 || sg.r >= R || sg.t0 < 0 || sg.t0 >= sg.t1 || sg.t1 > T) {
        std::printf("R=%d T=%d G=%d: CTA %d segment %d out of range (r %d, tiles %d..%d)\n", R, T, G, c, k, sg.r,
                    sg.t0, sg.t1);
        return 1;
      }
      if (sg.r < s.nb * G && (sg.t0 != 0 || sg.t1 != T || sg.r % G != c)) {
        std::printf("R=%d T=%d G=%d: band row block %d not whole on CTA %d\n", R, T, G, sg.r, c);
        return 1;
      }
      for (int t = sg.t0; t < sg.t1; ++t) {
        int& owner = cover[(size_t)sg.r * T + t];
        if (owner >= 0) {
          std::printf("R=%d T=%d G=%d: unit (%d, %d) covered twice\n", R, T, G, sg.r, t);
          return 1;
        }
        owner = c;
      }
      touch[(size_t)sg.r].push_back({c, k});
    }
  }
  for (int64_t u = 0; u < units; ++u)
    if (cover[(size_t)u] < 0) {
      std::printf("R=%d T=%d G=%d: unit %lld not covered\n", R, T, G, (long long)u);
      return 1;
    }
  for (int r = 0; r < R; ++r) {
    int cf = 0, cl = 0;
    progot::tc::contributors(s, r, &cf, &cl);
    const auto& tv = touch[(size_t)r];
    if ((int)tv.size() != cl - cf + 1) {
      std::printf("R=%d T=%d G=%d: row block %d has %zu segments, contributors %d..%d\n", R, T, G, r, tv.size(), cf,
                  cl);
      return 1;
    }
    for (size_t q = 0; q < tv.size(); ++q) {
      if (tv[q].first != cf + (int)q || progot::tc::seg_of(s, r, tv[q].first) != tv[q].second) {
        std::printf("R=%d T=%d G=%d: row block %d contributor %zu mismatch\n", R, T, G, r, q);
        return 1;
      }
    }
  }
  return 0;
}

int main() {
  const int Rs[] = {1, 2, 63, 64, 151, 152, 153, 157, 300, 304, 305, 469, 512, 1000};
  const int Ts[] = {1, 2, 3, 32, 33, 64, 235};
  const int Ss[] = {152, 148, 7, 1};
  int cases = 0;
  for (int R : Rs)
    for (int T : Ts)
      for (int sms : Ss) {
        if (check(R, T, sms)) return 1;
        ++cases;
      }
  uint64_t x = 0x9E3779B97F4A7C15ull;
  for (int i = 0; i < 400; ++i) {
    x ^= x << 13;
    x ^= x >> 7;
    x ^= x << 17;
    const int R = 1 + (int)(x % 1500), T = 1 + (int)((x >> 20) % 300), sms = 1 + (int)((x >> 40) % 200);
    if (check(R, T, sms)) return 1;
    ++cases;
  }
  std::printf("work split ok: %d cases\n", cases);
  return 0;
}
