// Request queue of the serving loop: tickets, FIFO admission by device-memory footprint,
// cancellation and completion.  Host-only C++17 (no CUDA): the serving workers in serve.cu
// take requests from it, and a host test drives it with fake work.
//
// Admission rule: requests are admitted in submission order; the request at the head of the
// queue is admitted when a worker is free and the footprints of the running requests plus its
// own fit the capacity.  A request whose footprint exceeds the whole capacity is refused at
// submission.  Later requests never overtake the head (no starvation of large requests).
#pragma once

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <memory>
#include <mutex>
#include <unordered_map>

namespace l1ls {

template <class Payload, class Outcome>
class AdmissionQueue {
public:
    enum State { kQueued, kRunning, kDone };
    using Clock = std::chrono::steady_clock;

    struct Request {
        uint64_t ticket = 0;
        size_t footprint = 0;
        State state = kQueued;
        bool cancelled = false;       // cancel() was called (queued: never runs; running: asked to stop)
        std::atomic<int> cancel_flag{0};   // polled by the work through cancel_requested()
        Payload payload{};
        Outcome outcome{};
        Clock::time_point t_submit, t_start, t_done;
    };
    using Ptr = std::shared_ptr<Request>;

    explicit AdmissionQueue(size_t capacity) : capacity_(capacity) {}

    size_t capacity() const { return capacity_; }

    // 0: refused (footprint above the capacity, or the queue is closed); else the ticket
    uint64_t submit(const Payload& p, size_t footprint) {
        std::lock_guard<std::mutex> lk(mu_);
        if (closed_ || footprint > capacity_) return 0;
        auto r = std::make_shared<Request>();
        r->ticket = next_++;
        r->footprint = footprint;
        r->payload = p;
        r->t_submit = Clock::now();
        queue_.push_back(r);
        all_[r->ticket] = r;
        work_cv_.notify_all();
        return r->ticket;
    }

    // Worker side: blocks until the head request is admissible (returns it, now running) or
    // the queue is closed (returns nullptr).
    Ptr acquire() {
        std::unique_lock<std::mutex> lk(mu_);
        for (;;) {
            drop_cancelled_head();
            if (closed_) return nullptr;
            if (!queue_.empty() && reserved_ + queue_.front()->footprint <= capacity_) {
                Ptr r = queue_.front();
                queue_.pop_front();
                r->state = kRunning;
                r->t_start = Clock::now();
                reserved_ += r->footprint;
                ++running_;
                if (running_ > peak_running_) peak_running_ = running_;
                if (reserved_ > peak_reserved_) peak_reserved_ = reserved_;
                return r;
            }
            work_cv_.wait(lk);
        }
    }

    // Worker side: the request finished (or stopped) with this outcome.
    void complete(const Ptr& r, const Outcome& out) {
        std::lock_guard<std::mutex> lk(mu_);
        r->outcome = out;
        r->state = kDone;
        r->t_done = Clock::now();
        reserved_ -= r->footprint;
        --running_;
        ++completed_;
        work_cv_.notify_all();
        done_cv_.notify_all();
    }

    // Poller side: waits up to wait_ms for the request to finish.  Returns nullptr for an
    // unknown ticket; otherwise the request (check its state).  A finished request is removed
    // (its ticket becomes unknown) when `consume` is set.
    Ptr wait(uint64_t ticket, int wait_ms, bool consume) {
        std::unique_lock<std::mutex> lk(mu_);
        auto it = all_.find(ticket);
        if (it == all_.end()) return nullptr;
        Ptr r = it->second;
        const auto until = Clock::now() + std::chrono::milliseconds(wait_ms > 0 ? wait_ms : 0);
        while (r->state != kDone && !(r->cancelled && r->state == kQueued)) {
            if (wait_ms <= 0 || done_cv_.wait_until(lk, until) == std::cv_status::timeout) break;
        }
        const bool finished = r->state == kDone || (r->cancelled && r->state == kQueued);
        if (finished && consume) all_.erase(ticket);
        return r;
    }

    // Cancel: a queued request is dropped, a running one is asked to stop.  false: unknown.
    bool cancel(uint64_t ticket) {
        std::lock_guard<std::mutex> lk(mu_);
        auto it = all_.find(ticket);
        if (it == all_.end()) return false;
        Ptr r = it->second;
        r->cancelled = true;
        if (r->state == kRunning) r->cancel_flag.store(1, std::memory_order_relaxed);
        work_cv_.notify_all();
        done_cv_.notify_all();
        return true;
    }

    // Close: refuse new submissions, cancel everything queued or running, wake all waiters.
    void close() {
        std::lock_guard<std::mutex> lk(mu_);
        closed_ = true;
        for (auto& kv : all_) {
            kv.second->cancelled = true;
            if (kv.second->state == kRunning) kv.second->cancel_flag.store(1, std::memory_order_relaxed);
        }
        work_cv_.notify_all();
        done_cv_.notify_all();
    }

    struct Stats {
        uint64_t completed;
        int running, peak_running;
        size_t reserved, peak_reserved;
        size_t queued;
    };
    Stats stats() {
        std::lock_guard<std::mutex> lk(mu_);
        return Stats{completed_, running_, peak_running_, reserved_, peak_reserved_, queue_.size()};
    }

    // the cancel flag of a running request, read without the lock by the work itself
    static bool cancel_requested(const Request& r) {
        return r.cancel_flag.load(std::memory_order_relaxed) != 0;
    }

private:
    void drop_cancelled_head() {
        while (!queue_.empty() && queue_.front()->cancelled) queue_.pop_front();
    }

    std::mutex mu_;
    std::condition_variable work_cv_, done_cv_;
    std::deque<Ptr> queue_;
    std::unordered_map<uint64_t, Ptr> all_;
    size_t capacity_;
    size_t reserved_ = 0, peak_reserved_ = 0;
    int running_ = 0, peak_running_ = 0;
    uint64_t completed_ = 0;
    uint64_t next_ = 1;
    bool closed_ = false;
};

}  // namespace l1ls
