// Host test of the serving loop's admission queue (no GPU): worker threads run fake work
// of known footprint and duration; the checks are the admission rule (submission order,
// running footprints within the capacity, no overtaking of the head), refusal, cancellation
// of queued and running requests, polling with a timeout, and shutdown.
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <mutex>
#include <thread>
#include <vector>

#include "serve_queue.h"

using namespace l1ls;
using namespace std::chrono;

struct Work {
    int ms;        // duration of the fake work
    int id;
};
struct Result {
    int id = -1;
    bool stopped = false;   // the work saw its cancel flag
};
using Q = AdmissionQueue<Work, Result>;

static int failures = 0;
#define CHECK(c)                                                       \
    do {                                                               \
        if (!(c)) {                                                    \
            std::fprintf(stderr, "FAILED line %d: %s\n", __LINE__, #c); \
            ++failures;                                                \
        }                                                              \
    } while (0)

struct Log {
    std::mutex mu;
    std::vector<int> start_order;
    size_t max_reserved = 0;
    size_t reserved = 0;
};

static void worker(Q* q, Log* log) {
    while (Q::Ptr r = q->acquire()) {
        {
            std::lock_guard<std::mutex> g(log->mu);
            log->start_order.push_back(r->payload.id);
            log->reserved += r->footprint;
            if (log->reserved > log->max_reserved) log->max_reserved = log->reserved;
        }
        Result out;
        out.id = r->payload.id;
        const auto until = steady_clock::now() + milliseconds(r->payload.ms);
        while (steady_clock::now() < until) {
            if (Q::cancel_requested(*r)) {
                out.stopped = true;
                break;
            }
            std::this_thread::sleep_for(milliseconds(1));
        }
        {
            std::lock_guard<std::mutex> g(log->mu);
            log->reserved -= r->footprint;
        }
        q->complete(r, out);
    }
}

static void test_admission_order_and_capacity() {
    Q q(100);
    Log log;
    // the 50 must wait for the 60; the 30 and 10 behind it must not overtake it
    const size_t fp[] = {60, 50, 30, 10, 40, 40, 20};
    std::vector<uint64_t> t;
    for (int i = 0; i < 7; ++i) t.push_back(q.submit(Work{40, i}, fp[i]));
    for (uint64_t k : t) CHECK(k != 0);
    std::vector<std::thread> ws;
    for (int i = 0; i < 4; ++i) ws.emplace_back(worker, &q, &log);
    std::vector<Q::Ptr> done;
    for (int i = 0; i < 7; ++i) {
        Q::Ptr r = q.wait(t[i], 5000, true);
        CHECK(r && r->state == Q::kDone && r->outcome.id == i);
        done.push_back(r);
    }
    CHECK(log.start_order.size() == 7);
    // admitted in submission order (admission times are taken under the queue's lock)
    for (int i = 0; i + 1 < 7; ++i) CHECK(done[i] && done[i + 1] && done[i]->t_start <= done[i + 1]->t_start);
    // the 50 started only after the 60 had finished
    CHECK(done[1]->t_start >= done[0]->t_done);
    CHECK(log.max_reserved <= 100);
    const Q::Stats s = q.stats();
    CHECK(s.completed == 7 && s.running == 0 && s.reserved == 0 && s.peak_reserved <= 100);
    CHECK(s.peak_running >= 2);                  // 50 + 30 + 10 ran together after the 60
    CHECK(q.wait(t[0], 0, true) == nullptr);     // consumed tickets are unknown
    q.close();
    for (auto& w : ws) w.join();
}

static void test_refusal_and_timeouts() {
    Q q(100);
    CHECK(q.submit(Work{1, 0}, 101) == 0);
    const uint64_t a = q.submit(Work{1, 1}, 100);
    CHECK(a != 0);
    // nobody runs it: a poll with a timeout returns it unfinished and keeps the ticket
    const auto t0 = steady_clock::now();
    Q::Ptr r = q.wait(a, 30, true);
    CHECK(r && r->state == Q::kQueued);
    CHECK(steady_clock::now() - t0 >= milliseconds(25));
    CHECK(q.wait(a, 0, true) != nullptr);
    CHECK(q.wait(12345, 0, true) == nullptr);
    q.close();
    CHECK(q.submit(Work{1, 2}, 1) == 0);         // closed
}

static void test_cancel() {
    Q q(100);
    Log log;
    const uint64_t big = q.submit(Work{2000, 0}, 80);     // runs, then is cancelled
    const uint64_t queued = q.submit(Work{10, 1}, 80);    // cannot fit next to it: stays queued
    const uint64_t after = q.submit(Work{10, 2}, 10);     // behind the queued head
    std::thread w1(worker, &q, &log), w2(worker, &q, &log);
    std::this_thread::sleep_for(milliseconds(50));
    CHECK(q.cancel(queued));
    Q::Ptr rq = q.wait(queued, 0, true);
    CHECK(rq && rq->state == Q::kQueued && rq->cancelled);
    CHECK(q.cancel(big));
    Q::Ptr rb = q.wait(big, 5000, true);
    CHECK(rb && rb->state == Q::kDone && rb->outcome.stopped);
    CHECK(duration_cast<milliseconds>(rb->t_done - rb->t_start).count() < 1500);
    Q::Ptr ra = q.wait(after, 5000, true);
    CHECK(ra && ra->state == Q::kDone && !ra->outcome.stopped);
    {
        std::lock_guard<std::mutex> g(log.mu);
        for (int id : log.start_order) CHECK(id != 1);     // the cancelled request never ran
    }
    CHECK(!q.cancel(999));
    q.close();
    w1.join();
    w2.join();
}

static void test_close_wakes_everyone() {
    Q q(10);
    std::atomic<int> returned{0};
    std::vector<std::thread> ws;
    for (int i = 0; i < 3; ++i)
        ws.emplace_back([&] {
            if (!q.acquire()) ++returned;
        });
    std::this_thread::sleep_for(milliseconds(20));
    q.close();
    for (auto& w : ws) w.join();
    CHECK(returned == 3);
}

int main() {
    test_admission_order_and_capacity();
    test_refusal_and_timeouts();
    test_cancel();
    test_close_wakes_everyone();
    if (failures) {
        std::fprintf(stderr, "%d check(s) failed\n", failures);
        return 1;
    }
    std::printf("OK\n");
    return 0;
}
