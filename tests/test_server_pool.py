"""The render server's framebuffer pool (csrc/gf_pool.h, host code), on the CPU:
random allocations and releases against a brute-force model of the free space."""
import os
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <cstdio>
#include <cstdlib>
#include <vector>
#include "gf_pool.h"

// brute force: one flag per 256-byte block; first fit = the lowest run of free
// blocks at least as long as the request
static bool model_alloc(std::vector<char>& used, size_t blocks, size_t& at) {
  size_t run = 0;
  for (size_t i = 0; i < used.size(); ++i) {
    run = used[i] ? 0 : run + 1;
    if (run == blocks) {
      at = i + 1 - blocks;
      for (size_t k = at; k <= i; ++k) used[k] = 1;
      return true;
    }
  }
  return false;
}

int main() {
  const size_t B = 256, total = 64 * B;
  gf::Pool pool;
  pool.init(total);
  std::vector<char> used(total / B, 0);
  struct A { size_t off, bytes; };
  std::vector<A> live;
  srand(7);
  for (int step = 0; step < 20000; ++step) {
    if (live.empty() || rand() % 3) {
      const size_t blocks = 1 + rand() % 12;
      size_t off = 0, at = 0;
      const bool got = pool.alloc(blocks * B, off);
      const bool want = model_alloc(used, blocks, at);
      if (got != want || (got && off != at * B)) {
        printf("alloc mismatch at step %d: %d %d %zu %zu\n", step, got, want, off, at * B);
        return 1;
      }
      if (got) live.push_back({off, blocks * B});
    } else {
      const size_t k = rand() % live.size();
      pool.release(live[k].off, live[k].bytes);
      for (size_t b = live[k].off / B; b < (live[k].off + live[k].bytes) / B; ++b) used[b] = 0;
      live[k] = live.back();
      live.pop_back();
    }
    size_t in_use = 0, free_bytes = 0, prev_end = 0;
    bool first = true;
    for (const A& a : live) in_use += a.bytes;
    for (const auto& kv : pool.free_blocks()) {
      // free blocks are disjoint, never adjacent (merged), and free in the model
      if (!first && kv.first <= prev_end) { printf("unmerged or overlapping free blocks\n"); return 1; }
      for (size_t b = kv.first / B; b < (kv.first + kv.second) / B; ++b)
        if (used[b]) { printf("free block over a live allocation\n"); return 1; }
      free_bytes += kv.second;
      prev_end = kv.first + kv.second;
      first = false;
    }
    if (pool.used() != in_use || in_use + free_bytes != total) {
      printf("byte count mismatch at step %d\n", step);
      return 1;
    }
  }
  for (const A& a : live) pool.release(a.off, a.bytes);
  if (pool.free_blocks().size() != 1 || pool.free_blocks().begin()->second != total) {
    printf("not merged back into one block\n");
    return 1;
  }
  printf("ok\n");
  return 0;
}
"""


def test_pool_first_fit_and_merging(tmp_path):
    src = tmp_path / "pool.cpp"
    src.write_text(PROGRAM)
    exe = tmp_path / "pool"
    subprocess.run(["g++", "-std=c++17", "-O1", "-I",
                    os.path.join(ROOT, "paper_2602_05081_gb300", "csrc"), str(src), "-o", str(exe)],
                   check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout
