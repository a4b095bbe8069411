"""The serving loop's device-arena allocator (csrc/cvs_arena.h), exercised on
the host: a randomized alloc/release sequence checked against a reference
model for overlap, alignment, accounting and coalescing (no GPU)."""
import subprocess
from pathlib import Path

ROOT = Path(__file__).resolve().parent.parent

PROGRAM = r'''
#include "cvs_arena.h"
#include <cstdio>
#include <cstdlib>
#include <map>
#include <random>
int main() {
    const int64_t size = 1 << 24;
    cvs::Arena a(size);
    std::mt19937_64 rng(7);
    std::map<int64_t, int64_t> live;  // offset -> requested bytes
    for (int it = 0; it < 200000; ++it) {
        if (live.empty() || rng() % 3 != 0) {
            const int64_t want = 1 + (int64_t)(rng() % 300000);
            const int64_t off = a.alloc(want);
            if (off < 0) {
                // must really be out of room for a block of this size
                if (a.largest_free() >= (want + 255) / 256 * 256) { std::puts("spurious failure"); return 1; }
                continue;
            }
            if (off % 256) { std::puts("misaligned"); return 1; }
            if (off + want > size) { std::puts("out of range"); return 1; }
            auto next = live.lower_bound(off);
            if (next != live.end() && next->first < off + want) { std::puts("overlap"); return 1; }
            if (next != live.begin()) {
                auto prev = std::prev(next);
                if (prev->first + prev->second > off) { std::puts("overlap"); return 1; }
            }
            live[off] = want;
        } else {
            auto it2 = live.begin();
            std::advance(it2, rng() % live.size());
            if (!a.release(it2->first)) { std::puts("release failed"); return 1; }
            live.erase(it2);
        }
        int64_t used = 0;
        for (auto& kv : live) used += (kv.second + 255) / 256 * 256;
        if (used != a.in_use()) { std::puts("accounting"); return 1; }
    }
    for (auto& kv : live) a.release(kv.first);
    if (a.in_use() != 0 || a.free_blocks() != 1 || a.largest_free() != size) {
        std::puts("not coalesced"); return 1;
    }
    if (a.release(12345)) { std::puts("released a non-block"); return 1; }
    std::puts("ok");
    return 0;
}
'''


def test_arena_randomized(tmp_path):
    src = tmp_path / "arena_test.cpp"
    src.write_text(PROGRAM)
    exe = tmp_path / "arena_test"
    subprocess.run(["g++", "-O2", "-std=c++17", "-I",
                    str(ROOT / "paper_2507_22901_gb300" / "csrc"), str(src), "-o", str(exe)],
                   check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout
