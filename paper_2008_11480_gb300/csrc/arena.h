// First-fit allocator of byte ranges inside one device allocation (the
// request workspaces of the continuous-batching server).  Host-only code:
// offsets in [0, size), 256-byte granules, neighbouring free ranges merged.
#pragma once
#include <cstddef>
#include <cstdint>
#include <iterator>
#include <map>

namespace nsgb {

struct Arena {
  std::map<size_t, size_t> free_;  // offset -> length
  size_t free_bytes() const {
    size_t t = 0;
    for (const auto& f : free_) t += f.second;
    return t;
  }
  void init(size_t s) {
    free_.clear();
    if (s) free_[0] = s;
  }
  size_t alloc(size_t bytes) {
    bytes = (bytes + 255) / 256 * 256;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      const size_t off = it->first, len = it->second;
      free_.erase(it);
      if (len > bytes) free_[off + bytes] = len - bytes;
      return off;
    }
    return SIZE_MAX;
  }
  void release(size_t off, size_t bytes) {
    bytes = (bytes + 255) / 256 * 256;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
};

}  // namespace nsgb
