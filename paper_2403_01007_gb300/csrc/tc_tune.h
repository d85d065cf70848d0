// Launch-shape choices of the persistent tensor-core contraction and the
// table that records the fastest choice per contraction shape.
//
// A contraction C (=, +=) alpha A B^T of M x N over nk K blocks can be run
// with either kernel variant (four epilogue warps and four pipeline stages, or
// eight epilogue warps and three stages, the latter only for at most four K
// blocks per work item), with the work items walked M-fastest or N-fastest,
// and with K split over 1..nk/4 extra work items whose partial results are
// summed afterwards. The default is a fixed rule of thumb; when tuning is on,
// the first contraction of each shape times every candidate and the table
// keeps the fastest for the rest of the process. The table is shared by all
// contexts and can be exported and imported as text.
//
// This file is plain C++ (no CUDA) so that the candidate rules and the text
// format are compiled and tested without a GPU as well.
#pragma once

#include <cstdint>
#include <mutex>
#include <string>
#include <map>
#include <tuple>
#include <vector>

namespace sccsd {

struct TcConfig {
  int variant = 0;   // 0: 4 epilogue warps, 4 stages; 1: 8 epilogue warps, 3 stages
  int nfast = 0;     // work-item order: 0 M tiles fastest, 1 N tiles fastest
  int splits = 1;    // K ranges per output tile
  int kbs = 1;       // K blocks per range (the last range may be shorter)
};

// Shape of one contraction as the tensor-core path sees it. view_hash
// identifies the output view (levels and strides), accumulate whether the
// epilogue reads the old values.
struct TcShape {
  int64_t M = 0, n_pad = 0;
  int nk = 0, slices = 1, accumulate = 0, sm_count = 0;
  uint64_t view_hash = 0;
  bool operator<(const TcShape& o) const {
    return std::tie(M, n_pad, nk, slices, accumulate, sm_count, view_hash) <
           std::tie(o.M, o.n_pad, o.nk, o.slices, o.accumulate, o.sm_count, o.view_hash);
  }
};

// The fixed rule: split K when the output tiles cannot fill the GPU (at least
// four K blocks per range), take N fastest when A is the larger operand, and
// the eight-warp variant for at most four K blocks per item.
TcConfig tc_default_config(const TcShape& s, int64_t m_tiles, int64_t n_tiles, double a_bytes,
                           double b_bytes);

// Every configuration the library launches for this shape (the default first).
std::vector<TcConfig> tc_candidates(const TcShape& s, int64_t m_tiles, int64_t n_tiles,
                                    double a_bytes, double b_bytes);

// Whether cfg is one of the forms the library launches for nk K blocks.
bool tc_config_valid(const TcConfig& cfg, int nk, int64_t n_tiles);

class TcTuneTable {
 public:
  static TcTuneTable& global();
  bool find(const TcShape& s, TcConfig& cfg) const;
  void put(const TcShape& s, const TcConfig& cfg, double us);
  size_t size() const;
  void clear();
  // one line per entry:
  //   M n_pad nk slices accumulate sm_count view_hash variant nfast splits kbs us
  std::string dump() const;
  // merge the entries of text written by dump(); on a malformed or invalid
  // line nothing is merged and the line number is returned (0 on success)
  int load(const std::string& text);

 private:
  struct Entry {
    TcConfig cfg;
    double us = 0.0;
  };
  mutable std::mutex mu_;
  std::map<TcShape, Entry> map_;
};

}  // namespace sccsd
