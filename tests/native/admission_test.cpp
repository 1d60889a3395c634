// CPU test of the render server's admission order (paper_2603_02048_gb300/
// csrc/admission.h): the order on hand-made cases, and on random queues
// against what the policy promises: younger requests smallest first, every
// request past the age limit ahead of every younger one and oldest first
// among those, equal keys in submission order, and no request admitted later
// than the age limit plus the requests that were ahead of it then.
#include <algorithm>
#include <cstdio>
#include <random>
#include <vector>

#include "admission.h"

#define CHECK(c)                                                  \
    do {                                                          \
        if (!(c)) {                                               \
            std::printf("FAIL line %d: %s\n", __LINE__, #c);      \
            return 1;                                             \
        }                                                         \
    } while (0)

struct Req {
    int id;
    hh::Waiting w;
};

static std::vector<int> order(std::vector<Req> q, double now, double age) {
    std::stable_sort(q.begin(), q.end(), [&](const Req& a, const Req& b) {
        return hh::admit_before(a.w, b.w, now, age);
    });
    std::vector<int> ids;
    for (const Req& r : q) ids.push_back(r.id);
    return ids;
}

int main() {
    const double age = 50.0;
    // young requests: fewest rays first, ties in submission order
    {
        std::vector<Req> q = {{0, {100.0, 900}}, {1, {101.0, 300}}, {2, {102.0, 300}},
                              {3, {103.0, 100}}};
        CHECK((order(q, 120.0, age) == std::vector<int>{3, 1, 2, 0}));
    }
    // a request past the age limit goes first, however large
    {
        std::vector<Req> q = {{0, {10.0, 1000000}}, {1, {100.0, 10}}, {2, {101.0, 5}}};
        CHECK((order(q, 70.0, age) == std::vector<int>{0, 2, 1}));
        // not yet past it (exactly at the limit): smallest first
        CHECK((order(q, 60.0, age) == std::vector<int>{2, 1, 0}));
    }
    // several past the limit: oldest first among them, then the young ones
    {
        std::vector<Req> q = {{0, {30.0, 7}}, {1, {10.0, 9000}}, {2, {95.0, 1}},
                              {3, {20.0, 50}}};
        CHECK((order(q, 100.0, age) == std::vector<int>{1, 3, 0, 2}));
    }
    // random queues: the promised structure
    std::mt19937_64 rng(12345);
    for (int trial = 0; trial < 2000; ++trial) {
        const int n = 1 + static_cast<int>(rng() % 40);
        const double now = 1000.0;
        std::vector<Req> q;
        for (int i = 0; i < n; ++i) {
            const double t = now - static_cast<double>(rng() % 120000) / 1000.0;  // 0-120 ms ago
            const uint64_t rays = 1 + rng() % 8;  // few distinct sizes: many ties
            q.push_back({i, {t, rays}});
        }
        const std::vector<int> ids = order(q, now, age);
        CHECK(static_cast<int>(ids.size()) == n);
        bool seen_young = false;
        for (int k = 0; k < n; ++k) {
            const Req& r = q[ids[k]];
            const bool old = now - r.w.t_submit > age;
            CHECK(!(old && seen_young));  // every old request before every young one
            seen_young |= !old;
            if (k + 1 < n) {
                const Req& s = q[ids[k + 1]];
                const bool old_s = now - s.w.t_submit > age;
                if (old && old_s) CHECK(r.w.t_submit <= s.w.t_submit);
                if (!old && !old_s) CHECK(r.w.rays <= s.w.rays);
                // equal keys keep submission order (the queue is in id order)
                if (old == old_s && r.w.t_submit == s.w.t_submit && r.w.rays == s.w.rays)
                    CHECK(r.id < s.id);
                if (!old && !old_s && r.w.rays == s.w.rays) CHECK(r.id < s.id);
            }
        }
    }
    // no starvation: a large request submitted at t0 among a stream of small
    // ones is admitted at the first admission after t0 + age (one request
    // admitted per ms, a new small one arriving every ms)
    {
        std::vector<Req> q = {{0, {0.0, 1000000}}};
        int next = 1;
        double admitted_at = -1.0;
        for (int ms = 1; ms <= 200 && admitted_at < 0; ++ms) {
            q.push_back({next++, {static_cast<double>(ms), 1}});
            const std::vector<int> ids = order(q, ms, age);
            const int first = ids[0];
            if (first == 0) admitted_at = ms;
            q.erase(std::find_if(q.begin(), q.end(), [&](const Req& r) { return r.id == first; }));
        }
        CHECK(admitted_at == 51.0);
    }
    std::printf("admission ok\n");
    return 0;
}
