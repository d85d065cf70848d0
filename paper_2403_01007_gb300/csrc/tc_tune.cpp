// Launch-shape candidates of the tensor-core contraction and the table of
// tuned choices (plain C++, shared by the device library and the host tests).
#include "tc_tune.h"

#include <algorithm>
#include <cstdio>
#include <sstream>

namespace sccsd {

namespace {

// K split into `want` ranges: ranges of ceil(nk / want) blocks
void split_of(int nk, int64_t want, TcConfig& c) {
  if (want <= 1) {
    c.splits = 1;
    c.kbs = nk;
    return;
  }
  c.kbs = (int)((nk + want - 1) / want);
  c.splits = (nk + c.kbs - 1) / c.kbs;
}

bool same(const TcConfig& a, const TcConfig& b) {
  return a.variant == b.variant && a.nfast == b.nfast && a.splits == b.splits && a.kbs == b.kbs;
}

}  // namespace

TcConfig tc_default_config(const TcShape& s, int64_t m_tiles, int64_t n_tiles, double a_bytes,
                           double b_bytes) {
  TcConfig c;
  const int64_t tiles = m_tiles * n_tiles;
  int64_t want = 1;
  if (tiles < s.sm_count && s.nk >= 8)
    want = std::min<int64_t>((2 * (int64_t)s.sm_count + tiles - 1) / tiles, s.nk / 4);
  // split only when it shortens the work per SM: waves of the split grid per
  // unit of work at most 0.85 of the unsplit grid's (a grid that already
  // fills most SMs in one wave gains nothing and pays for the reduction)
  if (want > 1) {
    const int64_t sms = s.sm_count;
    const double w1 = (double)((tiles + sms - 1) / sms);
    const double ws = (double)((want * tiles + sms - 1) / sms) / (double)want;
    if (ws > 0.85 * w1) want = 1;
  }
  split_of(s.nk, want, c);
  c.nfast = (n_tiles > 1 && a_bytes > 4.0 * b_bytes) ? 1 : 0;
  // eight epilogue warps (three pipeline stages) when an item has at most 16
  // K blocks: its MMAs then take no longer than its FP64 epilogue
  c.variant = c.kbs <= 16 ? 1 : 0;
  return c;
}

std::vector<TcConfig> tc_candidates(const TcShape& s, int64_t m_tiles, int64_t n_tiles,
                                    double a_bytes, double b_bytes) {
  const TcConfig d = tc_default_config(s, m_tiles, n_tiles, a_bytes, b_bytes);
  std::vector<TcConfig> out{d};
  std::vector<int64_t> wants{1};
  if (s.nk >= 8) {
    const int64_t maxw = s.nk / 4, dw = d.splits;
    for (int64_t w : {dw, dw / 2, 2 * dw, maxw})
      if (w >= 2 && w <= maxw) wants.push_back(w);
  }
  for (int64_t w : wants) {
    TcConfig c;
    split_of(s.nk, w, c);
    for (int variant = 0; variant < 2; ++variant) {
      for (int nfast = 0; nfast < (n_tiles > 1 ? 2 : 1); ++nfast) {
        TcConfig x = c;
        x.variant = variant;
        x.nfast = nfast;
        bool dup = false;
        for (const TcConfig& y : out) dup = dup || same(x, y);
        if (!dup) out.push_back(x);
      }
    }
  }
  return out;
}

bool tc_config_valid(const TcConfig& c, int nk, int64_t n_tiles) {
  if (nk < 1 || c.variant < 0 || c.variant > 1 || c.nfast < 0 || c.nfast > 1) return false;
  if (c.nfast == 1 && n_tiles < 2) return false;
  if (c.splits == 1) {
    if (c.kbs != nk) return false;
  } else {
    if (c.splits < 1 || nk < 8 || c.kbs < 4 || c.splits != (nk + c.kbs - 1) / c.kbs) return false;
  }
  return true;
}

TcTuneTable& TcTuneTable::global() {
  static TcTuneTable t;
  return t;
}

bool TcTuneTable::find(const TcShape& s, TcConfig& cfg) const {
  std::lock_guard<std::mutex> g(mu_);
  auto it = map_.find(s);
  if (it == map_.end()) return false;
  cfg = it->second.cfg;
  return true;
}

void TcTuneTable::put(const TcShape& s, const TcConfig& cfg, double us) {
  std::lock_guard<std::mutex> g(mu_);
  map_[s] = Entry{cfg, us};
}

size_t TcTuneTable::size() const {
  std::lock_guard<std::mutex> g(mu_);
  return map_.size();
}

void TcTuneTable::clear() {
  std::lock_guard<std::mutex> g(mu_);
  map_.clear();
}

std::string TcTuneTable::dump() const {
  std::lock_guard<std::mutex> g(mu_);
  std::ostringstream os;
  for (const auto& kv : map_) {
    const TcShape& s = kv.first;
    const TcConfig& c = kv.second.cfg;
    char line[256];
    std::snprintf(line, sizeof line, "%lld %lld %d %d %d %d %llu %d %d %d %d %.3f\n",
                  (long long)s.M, (long long)s.n_pad, s.nk, s.slices, s.accumulate, s.sm_count,
                  (unsigned long long)s.view_hash, c.variant, c.nfast, c.splits, c.kbs,
                  kv.second.us);
    os << line;
  }
  return os.str();
}

int TcTuneTable::load(const std::string& text) {
  std::vector<std::pair<TcShape, Entry>> parsed;
  std::istringstream is(text);
  std::string line;
  int lineno = 0;
  while (std::getline(is, line)) {
    ++lineno;
    if (line.find_first_not_of(" \t\r") == std::string::npos) continue;
    std::istringstream ls(line);
    TcShape s;
    Entry e;
    long long M = 0, n_pad = 0;
    unsigned long long h = 0;
    std::string rest;
    if (!(ls >> M >> n_pad >> s.nk >> s.slices >> s.accumulate >> s.sm_count >> h >> e.cfg.variant >>
          e.cfg.nfast >> e.cfg.splits >> e.cfg.kbs >> e.us) ||
        (ls >> rest))
      return lineno;
    s.M = M;
    s.n_pad = n_pad;
    s.view_hash = h;
    const int64_t n_tiles = n_pad / 256;
    if (M < 1 || n_pad < 256 || n_pad % 256 != 0 || s.slices < 1 || s.slices > 2 ||
        (s.accumulate != 0 && s.accumulate != 1) || s.sm_count < 1 ||
        !tc_config_valid(e.cfg, s.nk, n_tiles))
      return lineno;
    parsed.push_back({s, e});
  }
  std::lock_guard<std::mutex> g(mu_);
  for (auto& p : parsed) map_[p.first] = p.second;
  return 0;
}

}  // namespace sccsd
