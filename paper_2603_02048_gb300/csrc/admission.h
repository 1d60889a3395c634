// Admission order of the render server's waiting requests (host logic only).
// Requests are taken smallest first (fewest rays), so short requests are not
// stuck behind large ones; a request that has waited longer than the age
// limit goes ahead of every younger one, oldest first among such requests,
// so a large request is delayed by at most the age limit plus the work
// admitted before it, never starved. Ties keep submission order (the caller
// sorts stably).
#pragma once

#include <cstdint>

namespace hh {

struct Waiting {
    double t_submit;  // ms on the server's clock
    uint64_t rays;    // pixels over all of the request's views
};

// Whether a is admitted before b at time now_ms.
inline bool admit_before(const Waiting& a, const Waiting& b, double now_ms, double age_ms) {
    const bool old_a = now_ms - a.t_submit > age_ms, old_b = now_ms - b.t_submit > age_ms;
    if (old_a != old_b) return old_a;
    if (old_a) return a.t_submit < b.t_submit;
    return a.rays < b.rays;
}

}  // namespace hh
