// Admission of likelihood requests to a pool of workers under an HBM budget
// (host logic only; no CUDA).  Used by the worker pool (pool.cu) and by the
// discrete-event simulator behind tlr_sched_simulate, which tests the policy
// without a GPU.
//
// Memory model.  Each dataset holds `base` bytes while it is registered
// (ordered locations, observations, permutation), `fbytes` while its TLR
// factor storage is resident, and a request of it holds `wbytes` of
// evaluation workspace while it runs.  `used` is the sum of those; the policy
// keeps used <= budget at all times.
//
// Policy.  Requests wait in one queue in arrival order.  admit() returns the
// earliest queued request that can start now:
//   - its dataset has no running request (the requests of one dataset run one
//     at a time, in arrival order, because each starts from the rank map the
//     previous one left);
//   - its workspace, plus its factor storage if that is not resident, fits:
//     idle resident factors of other datasets are evicted least recently used
//     first to make room;
//   - no earlier request is waiting for memory to allocate a factor when this
//     one would allocate one too (so a large dataset is not starved by a
//     stream of smaller ones).
#pragma once

#include <stdint.h>

#include <algorithm>
#include <deque>
#include <functional>
#include <vector>

namespace tlr {

class Admission {
public:
    struct Data {
        int64_t base = 0, fbytes = 0, wbytes = 0;
        bool alive = false, resident = false, busy = false;
        uint64_t last_use = 0;  // logical clock of the last finished request
    };
    struct Req {
        int64_t ticket;
        int data;
    };

    explicit Admission(int64_t budget = 0) : budget_(budget) {}

    int64_t budget() const { return budget_; }
    int64_t used() const { return used_; }
    int64_t peak() const { return peak_; }
    int64_t evictions() const { return evictions_; }
    size_t queued() const { return queue_.size(); }
    const Data &data(int d) const { return data_[(size_t)d]; }

    // Whether a dataset with these sizes can be registered: its base bytes
    // join every other dataset's, and every registered dataset (and this one)
    // must still be able to run alone with its factor and workspace.
    bool can_add(int64_t base, int64_t fbytes, int64_t wbytes) const {
        int64_t bases = base, worst = fbytes + wbytes;
        for (const Data &d : data_)
            if (d.alive) {
                bases += d.base;
                worst = std::max(worst, d.fbytes + d.wbytes);
            }
        return bases + worst <= budget_;
    }

    // Registers a dataset; returns its index (the caller checks can_add).
    int add(int64_t base, int64_t fbytes, int64_t wbytes) {
        Data d;
        d.base = base;
        d.fbytes = fbytes;
        d.wbytes = wbytes;
        d.alive = true;
        data_.push_back(d);
        charge(base);
        return (int)data_.size() - 1;
    }

    // Unregisters an idle dataset with no queued request; its base bytes and
    // resident factor are released.
    void remove(int d) {
        Data &x = data_[(size_t)d];
        if (x.resident) used_ -= x.fbytes;
        used_ -= x.base;
        x = Data();
    }

    // Whether dataset d could run alone with these factor / workspace sizes.
    bool resize_check(int d, int64_t fbytes, int64_t wbytes) const {
        (void)d;
        return bases() + fbytes + wbytes <= budget_;
    }

    // New factor / workspace sizes of an idle dataset whose factor is not
    // resident (a tile-size change); false (nothing changed) if they cannot
    // fit alone.
    bool resize(int d, int64_t fbytes, int64_t wbytes) {
        Data &x = data_[(size_t)d];
        if (x.resident || x.busy || !resize_check(d, fbytes, wbytes)) return false;
        x.fbytes = fbytes;
        x.wbytes = wbytes;
        return true;
    }

    // New workspace estimate of an idle dataset, capped so that the dataset
    // can still run alone (an uncapped estimate could never be admitted).
    void set_work(int d, int64_t wbytes) {
        Data &x = data_[(size_t)d];
        x.wbytes = std::max<int64_t>(0, std::min(wbytes, budget_ - bases() - x.fbytes));
    }

    // New factor size of a dataset whose factor is not resident (its next
    // allocation), capped like set_work so that it can still run alone.
    void set_factor(int d, int64_t fbytes) {
        Data &x = data_[(size_t)d];
        if (x.resident) return;
        x.fbytes = std::max<int64_t>(0, std::min(fbytes, budget_ - bases() - x.wbytes));
    }

    // Drops the resident factor of an idle dataset (returns whether it was resident).
    bool drop(int d) {
        Data &x = data_[(size_t)d];
        if (!x.resident || x.busy) return false;
        x.resident = false;
        used_ -= x.fbytes;
        return true;
    }

    void enqueue(int64_t ticket, int d) { queue_.push_back(Req{ticket, d}); }

    // Takes the next admissible request (see the policy above).  On success
    // *alloc says whether its factor storage must be allocated and `evicted`
    // receives the datasets whose factors were evicted to make room (their
    // storage must be freed by the caller before allocating).  With `only`,
    // requests for which it returns false are passed over (their datasets'
    // later requests too, which keeps each dataset's order); a worker that
    // evaluates several requests together takes its companions this way.
    bool admit(Req *out, bool *alloc, std::vector<int> *evicted,
               const std::function<bool(const Req &)> &only = nullptr) {
        bool mem_wait = false;
        seen_.assign(data_.size(), 0);
        for (auto it = queue_.begin(); it != queue_.end(); ++it) {
            const int d = it->data;
            Data &x = data_[(size_t)d];
            if (seen_[(size_t)d] || x.busy || (only && !only(*it))) {
                seen_[(size_t)d] = 1;
                continue;
            }
            seen_[(size_t)d] = 1;
            const bool need_alloc = !x.resident;
            if (need_alloc && mem_wait) continue;
            const int64_t need = x.wbytes + (need_alloc ? x.fbytes : 0);
            if (used_ + need > budget_) {
                int64_t idle = 0;
                for (size_t e = 0; e < data_.size(); ++e)
                    if ((int)e != d && data_[e].resident && !data_[e].busy) idle += data_[e].fbytes;
                if (used_ - idle + need > budget_) {
                    mem_wait = true;
                    continue;
                }
                while (used_ + need > budget_) {  // least recently used idle factor first
                    int victim = -1;
                    for (size_t e = 0; e < data_.size(); ++e)
                        if ((int)e != d && data_[e].resident && !data_[e].busy &&
                            (victim < 0 || data_[e].last_use < data_[(size_t)victim].last_use))
                            victim = (int)e;
                    data_[(size_t)victim].resident = false;
                    used_ -= data_[(size_t)victim].fbytes;
                    ++evictions_;
                    if (evicted) evicted->push_back(victim);
                }
            }
            charge(need);
            x.resident = true;
            x.busy = true;
            *out = *it;
            *alloc = need_alloc;
            queue_.erase(it);
            return true;
        }
        return false;
    }

    // Extra factor storage for the running request of dataset d (a retry on
    // larger slots): charged at once if it fits, else after evicting idle
    // factors of other datasets least recently used first.  Returns false if
    // it cannot fit now; *never then says whether it cannot fit even with every
    // other request finished and every idle factor evicted.
    bool grow(int d, int64_t extra, std::vector<int> *evicted, bool *never) {
        *never = false;
        if (extra <= 0) return true;
        const Data &x = data_[(size_t)d];
        if (bases() + x.fbytes + x.wbytes + extra > budget_) {
            *never = true;
            return false;
        }
        int64_t idle = 0;
        for (size_t e = 0; e < data_.size(); ++e)
            if ((int)e != d && data_[e].resident && !data_[e].busy) idle += data_[e].fbytes;
        if (used_ - idle + extra > budget_) return false;  // wait for running requests
        while (used_ + extra > budget_) {
            int victim = -1;
            for (size_t e = 0; e < data_.size(); ++e)
                if ((int)e != d && data_[e].resident && !data_[e].busy &&
                    (victim < 0 || data_[e].last_use < data_[(size_t)victim].last_use))
                    victim = (int)e;
            data_[(size_t)victim].resident = false;
            used_ -= data_[(size_t)victim].fbytes;
            ++evictions_;
            if (evicted) evicted->push_back(victim);
        }
        charge(extra);
        return true;
    }

    // Releases extra storage taken by grow().
    void shrink(int64_t extra) {
        if (extra > 0) used_ -= extra;
    }

    // The running request of dataset d has finished; `keep` false if its
    // factor storage was not kept (allocation failed).
    void finish(int d, bool keep = true) {
        Data &x = data_[(size_t)d];
        x.busy = false;
        x.last_use = ++clock_;
        used_ -= x.wbytes;
        if (!keep && x.resident) {
            x.resident = false;
            used_ -= x.fbytes;
        }
    }

private:
    int64_t bases() const {
        int64_t b = 0;
        for (const Data &y : data_)
            if (y.alive) b += y.base;
        return b;
    }
    void charge(int64_t b) {
        used_ += b;
        peak_ = std::max(peak_, used_);
    }

    int64_t budget_ = 0, used_ = 0, peak_ = 0, evictions_ = 0;
    uint64_t clock_ = 0;
    std::vector<Data> data_;
    std::deque<Req> queue_;
    std::vector<char> seen_;
};

}  // namespace tlr
