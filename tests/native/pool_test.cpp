// CPU test of the server's output-memory allocator (paper_2603_02048_gb300/
// csrc/pool.h): randomised alloc/release against a brute-force occupancy map.
#include <cstdio>
#include <cstdlib>
#include <map>
#include <random>
#include <vector>

#include "pool.h"

#define CHECK(c)                                                  \
    do {                                                          \
        if (!(c)) {                                               \
            std::printf("FAIL line %d: %s\n", __LINE__, #c);      \
            return 1;                                             \
        }                                                         \
    } while (0)

int main() {
    // basics
    hh::OffsetPool p(4096, 256);
    size_t a, b, c;
    CHECK(p.alloc(1, &a) && a == 0 && p.used() == 256);
    CHECK(p.alloc(300, &b) && b == 256 && p.used() == 768);
    CHECK(p.alloc(3328, &c) && c == 768 && p.used() == 4096);
    size_t d;
    CHECK(!p.alloc(1, &d));                 // full
    CHECK(p.release(b) && p.used() == 3584);
    CHECK(!p.release(b));                   // double free refused
    CHECK(!p.release(12345));               // unknown offset refused
    CHECK(p.alloc(512, &d) && d == 256);    // first fit reuses the hole
    CHECK(p.release(a) && p.release(c) && p.release(d));
    CHECK(p.used() == 0 && p.free_blocks() == 1 && p.largest_free() == 4096);
    CHECK(!p.alloc(4097, &d));              // larger than the capacity
    CHECK(!p.alloc(SIZE_MAX, &d));          // rounding overflow is refused
    CHECK(p.footprint(0) == 256 && p.footprint(257) == 512);

    // randomised against a byte-occupancy model
    std::mt19937_64 rng(7);
    const size_t cap = 1 << 20;
    hh::OffsetPool q(cap, 256);
    std::vector<char> owner(cap, 0);
    std::map<size_t, size_t> live;
    for (int it = 0; it < 200000; ++it) {
        if (live.empty() || rng() % 3) {
            const size_t want = 1 + rng() % 20000;
            size_t off;
            if (q.alloc(want, &off)) {
                const size_t n = q.footprint(want);
                CHECK(off % 256 == 0 && off + n <= cap);
                for (size_t i = off; i < off + n; ++i) CHECK(!owner[i]);
                for (size_t i = off; i < off + n; ++i) owner[i] = 1;
                live[off] = n;
            } else {
                // first fit failed: no free run of the rounded size exists
                const size_t n = q.footprint(want);
                size_t run = 0, best = 0;
                for (size_t i = 0; i < cap; i += 256) {
                    run = owner[i] ? 0 : run + 256;
                    best = run > best ? run : best;
                }
                CHECK(best < n);
            }
        } else {
            auto itl = live.begin();
            std::advance(itl, rng() % live.size());
            CHECK(q.release(itl->first));
            for (size_t i = itl->first; i < itl->first + itl->second; ++i) owner[i] = 0;
            live.erase(itl);
        }
        size_t used = 0;
        for (auto& kv : live) used += kv.second;
        CHECK(q.used() == used);
    }
    for (auto& kv : live) CHECK(q.release(kv.first));
    CHECK(q.used() == 0 && q.free_blocks() == 1 && q.largest_free() == cap);
    std::printf("pool ok\n");
    return 0;
}
