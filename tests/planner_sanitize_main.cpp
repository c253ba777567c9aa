// Drives the serving planner (admission and step planning, host-only) through
// seeded random request streams in a build with AddressSanitizer and
// UndefinedBehaviorSanitizer, and checks its invariants: the accounted bytes
// stay under the cap, no two admitted requests share a slot, requests are
// admitted in arrival order, and every tile of every request is planned
// exactly once, in order.  Exit status 0 when all hold.
#include <cstdio>
#include <map>
#include <random>
#include <set>
#include <vector>

#include "wt_planner.h"

int main() {
    int bad = 0;
    for (int trial = 0; trial < 200; ++trial) {
        std::mt19937_64 rng(1234 + trial);
        const int slots = 1 + (int)(rng() % 6);
        const int64_t cap = 1000 + (int64_t)(rng() % 5000);
        const int64_t step = 1 + (int64_t)(rng() % 64);
        wt::Planner p(slots, cap, step);
        std::map<int64_t, int64_t> tiles, next, bytes;
        std::vector<int64_t> order;  // arrival order of accepted requests
        std::set<int64_t> admitted_ids, live;
        size_t admitted_upto = 0;
        for (int round = 0; round < 300; ++round) {
            const int arrivals = (int)(rng() % 3);
            for (int a = 0; a < arrivals; ++a) {
                const int64_t b = (int64_t)(rng() % (uint64_t)(cap + 200));
                const int64_t t = (int64_t)(rng() % 50);
                const int64_t id = p.submit(b, t);
                if (b > cap) {
                    if (id != -(int64_t)WT_ERR_NOMEM) { std::printf("oversized request accepted\n"); bad = 1; }
                    continue;
                }
                tiles[id] = t;
                next[id] = 0;
                bytes[id] = b;
                order.push_back(id);
            }
            std::vector<int64_t> adm;
            p.admit(adm, [](int64_t) { return true; });
            for (int64_t id : adm) {
                if (admitted_upto >= order.size() || order[admitted_upto] != id) {
                    std::printf("admission out of arrival order\n");
                    bad = 1;
                }
                ++admitted_upto;
                admitted_ids.insert(id);
                live.insert(id);
            }
            std::set<int> used_slots;
            int64_t used = 0;
            for (int64_t id : live) {
                const int s = p.slot_of(id);
                if (s < 0 || s >= slots || !used_slots.insert(s).second) { std::printf("slot clash\n"); bad = 1; }
                used += bytes[id];
            }
            if (used != p.used() || used > cap) { std::printf("bytes %lld / %lld\n", (long long)used, (long long)p.used()); bad = 1; }
            std::vector<wt::Planner::Range> ranges;
            std::vector<int64_t> fin;
            p.plan(ranges, fin);
            int64_t planned = 0;
            for (const auto &r : ranges) {
                if (!live.count(r.id) || r.tile0 != next[r.id] || r.count <= 0) {
                    std::printf("bad range id %lld tile0 %d count %d\n", (long long)r.id, r.tile0, r.count);
                    bad = 1;
                }
                next[r.id] += r.count;
                planned += r.count;
            }
            if (planned > step) { std::printf("step over budget\n"); bad = 1; }
            for (int64_t id : fin) {
                if (next[id] != tiles[id]) { std::printf("finished early\n"); bad = 1; }
                if (p.release(id) != WT_OK) { std::printf("release refused\n"); bad = 1; }
                live.erase(id);
            }
            if (p.release(987654321) == WT_OK) { std::printf("unknown release accepted\n"); bad = 1; }
        }
        // drain: keep planning until every accepted request has finished
        for (int guard = 0; guard < 100000 && (p.queued() > 0 || p.active() > 0 || !live.empty()); ++guard) {
            std::vector<int64_t> adm;
            p.admit(adm, [](int64_t) { return true; });
            for (int64_t id : adm) live.insert(id);
            std::vector<wt::Planner::Range> ranges;
            std::vector<int64_t> fin;
            p.plan(ranges, fin);
            for (const auto &r : ranges) next[r.id] += r.count;
            for (int64_t id : fin) {
                p.release(id);
                live.erase(id);
            }
        }
        for (const auto &kv : tiles)
            if (next[kv.first] != kv.second) { std::printf("tiles planned %lld of %lld\n", (long long)next[kv.first], (long long)kv.second); bad = 1; }
        if (p.used() != 0) { std::printf("bytes left after drain\n"); bad = 1; }
    }
    if (!bad) std::printf("planner sanitizer run: ok\n");
    return bad;
}
