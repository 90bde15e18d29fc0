// gf_pool.h -- first-fit allocator of the render server's framebuffer pool
// (host code; offsets into one device allocation).  Blocks are 256-byte
// multiples and neighbouring free blocks are merged on release.
#pragma once
#include <cstddef>
#include <iterator>
#include <map>

namespace gf {

class Pool {
 public:
  void init(size_t bytes) {
    free_.clear();
    if (bytes) free_[0] = bytes;
    used_ = 0;
  }
  bool alloc(size_t bytes, size_t& off) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      off = it->first;
      const size_t rest = it->second - bytes;
      free_.erase(it);
      if (rest) free_[off + bytes] = rest;
      used_ += bytes;
      return true;
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    used_ -= bytes;
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
  size_t used() const { return used_; }
  const std::map<size_t, size_t>& free_blocks() const { return free_; }  // offset -> bytes

 private:
  std::map<size_t, size_t> free_;
  size_t used_ = 0;
};

}  // namespace gf
