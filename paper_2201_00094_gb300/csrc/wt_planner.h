// Admission and step planning of the serving runtime: host-only C++ with no
// CUDA dependency, so that it is tested on the CPU (through the library's
// wt_planner_* calls, and built alone under the address and undefined-behaviour
// sanitizers by the tests).
#pragma once
#include <stdint.h>

#include <algorithm>
#include <deque>
#include <unordered_map>
#include <vector>

#include "wt.h"

namespace wt {

class Planner {
  public:
    struct Range {
        int64_t id;
        int32_t slot, tile0, count;
    };

    Planner(int max_slots, int64_t cap, int64_t step_tiles)
        : max_slots_(max_slots), cap_(cap), step_tiles_(step_tiles) {
        for (int s = max_slots - 1; s >= 0; --s) free_slots_.push_back(s);
    }

    // Queues a request of `bytes` and `tiles`; returns its id, or -WT_ERR_NOMEM
    // when it could never fit under the cap.
    int64_t submit(int64_t bytes, int64_t tiles) {
        if (bytes > cap_ || bytes < 0 || tiles < 0) return -(int64_t)WT_ERR_NOMEM;
        const int64_t id = next_id_++;
        Req r;
        r.bytes = bytes;
        r.tiles = tiles;
        reqs_[id] = r;
        queue_.push_back(id);
        return id;
    }

    // Admits queued requests in arrival order while a slot and memory allow
    // (the head of the queue blocks the rest: no overtaking).  `fits`, when
    // given, is asked last (the server's arena allocation) and may refuse.
    template <class Fits> void admit(std::vector<int64_t> &admitted, Fits &&fits) {
        while (!queue_.empty()) {
            const int64_t id = queue_.front();
            Req &r = reqs_[id];
            if (free_slots_.empty() || used_ + r.bytes > cap_) break;
            if (!fits(id)) break;
            queue_.pop_front();
            r.slot = free_slots_.back();
            free_slots_.pop_back();
            r.state = kAdmitted;
            used_ += r.bytes;
            active_.push_back(id);
            admitted.push_back(id);
        }
    }

    // Plans one step: an equal share of the tile budget for every admitted
    // request with tiles left (leftover budget goes to the oldest first).
    // `finishing` lists requests whose last tiles are in this step.
    void plan(std::vector<Range> &ranges, std::vector<int64_t> &finishing) {
        int64_t budget = step_tiles_;
        std::vector<int64_t> live;
        for (int64_t id : active_)
            if (reqs_[id].next < reqs_[id].tiles) live.push_back(id);
        // one range per request and step: the second pass extends the first
        std::unordered_map<int64_t, size_t> at;
        for (int pass = 0; pass < 2 && budget > 0 && !live.empty(); ++pass) {
            const int64_t share = std::max<int64_t>(1, budget / (int64_t)live.size());
            for (int64_t id : live) {
                Req &r = reqs_[id];
                const int64_t left = r.tiles - r.next;
                const int64_t take = std::min({left, pass == 0 ? share : left, budget});
                if (take <= 0) continue;
                auto it = at.find(id);
                if (it == at.end()) {
                    at[id] = ranges.size();
                    ranges.push_back({id, r.slot, (int32_t)r.next, (int32_t)take});
                } else {
                    ranges[it->second].count += (int32_t)take;
                }
                r.next += take;
                budget -= take;
                if (budget <= 0) break;
            }
        }
        for (int64_t id : live) {
            Req &r = reqs_[id];
            if (r.next >= r.tiles && r.state == kAdmitted) {
                r.state = kScheduled;
                finishing.push_back(id);
            }
        }
        // requests with no tiles finish at once
        for (int64_t id : active_) {
            Req &r = reqs_[id];
            if (r.tiles == 0 && r.state == kAdmitted) {
                r.state = kScheduled;
                finishing.push_back(id);
            }
        }
        active_.erase(std::remove_if(active_.begin(), active_.end(),
                                     [&](int64_t id) { return reqs_[id].state != kAdmitted; }),
                      active_.end());
    }

    // Frees the request's slot and bytes (it must have been fully scheduled).
    wt_status release(int64_t id) {
        auto it = reqs_.find(id);
        if (it == reqs_.end() || it->second.state != kScheduled) return WT_ERR_ARG;
        used_ -= it->second.bytes;
        free_slots_.push_back(it->second.slot);
        reqs_.erase(it);
        return WT_OK;
    }

    int slot_of(int64_t id) const {
        auto it = reqs_.find(id);
        return it == reqs_.end() ? -1 : it->second.slot;
    }
    int64_t used() const { return used_; }
    int64_t queued() const { return (int64_t)queue_.size(); }
    int64_t active() const { return (int64_t)active_.size(); }
    bool known(int64_t id) const { return reqs_.count(id) != 0; }

  private:
    enum { kQueued = 0, kAdmitted = 1, kScheduled = 2 };
    struct Req {
        int64_t bytes = 0, tiles = 0, next = 0;
        int slot = -1;
        int state = kQueued;
    };
    int max_slots_;
    int64_t cap_, step_tiles_;
    int64_t used_ = 0, next_id_ = 1;
    std::deque<int64_t> queue_;
    std::vector<int64_t> active_;
    std::vector<int> free_slots_;
    std::unordered_map<int64_t, Req> reqs_;
};

}  // namespace wt
