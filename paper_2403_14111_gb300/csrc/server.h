// server.h -- continuous-batching request loop for encrypted matrix products.
//
// Clients register their evaluation keys (kept resident on the device) and
// submit DiagABT / DiagATB requests on ciphertexts already on the device.  A
// scheduler thread admits requests in arrival order whenever a slot (a worker
// thread with its own CUDA stream) is free and the request's estimated device
// footprint fits the memory budget beside the resident keys and the requests
// in flight; admitted requests run concurrently, so work that arrives while
// others are on the GPU overlaps with them.  Each request records its queueing
// and running time.
#pragma once
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <set>
#include <thread>

#include "runtime.h"

namespace hetal {

struct ServerRequest {
    int client = 0;
    int kind = 0;                 // 0 DiagABT(a, b = B-bar), 1 DiagATB(a = A-underbar, b = B)
    const Mat *a = nullptr, *b = nullptr;
    int c = 2;
    double t = 1.0;
    int flags = 0;
};

struct ServerResult {
    Mat out;
    int status = 0;
    std::string error;
    double queue_ms = 0, run_ms = 0;
    size_t footprint = 0;
};

class Server {
  public:
    Server(const Params &p, int device, int slots, size_t budget_bytes);
    ~Server();
    int add_client(const EvalKeys *ek, size_t key_bytes);
    uint64_t submit(const ServerRequest &r);
    // withdraws a queued request; false if it is not queued (unknown, running, done or taken)
    bool cancel(uint64_t ticket);
    // waits for a ticket; returns false if the ticket is unknown or already taken
    bool wait(uint64_t ticket, ServerResult &out);
    size_t resident_bytes() const { return resident_; }
    size_t peak_inflight_bytes() const { return peak_inflight_; }
    long long completed() const { return completed_; }

  private:
    struct Job {
        uint64_t ticket;
        ServerRequest req;
        size_t footprint;
        std::chrono::steady_clock::time_point submitted;
    };
    size_t estimate(const ServerRequest &r) const;
    void scheduler();
    void worker(int slot);

    std::vector<std::unique_ptr<Context>> ctxs_;
    std::vector<std::thread> workers_;
    std::thread sched_;
    std::mutex mu_;
    std::condition_variable cv_;        // scheduler: arrivals, completions
    std::condition_variable work_cv_;   // workers: dispatched jobs
    std::condition_variable done_cv_;   // waiters: completions
    std::deque<Job> pending_;
    std::vector<std::deque<Job>> assigned_;
    std::vector<bool> busy_;
    std::map<uint64_t, ServerResult> results_;
    std::set<uint64_t> taken_;
    std::map<int, const EvalKeys *> clients_;
    size_t budget_, resident_ = 0, inflight_ = 0, peak_inflight_ = 0;
    long long completed_ = 0;
    uint64_t next_ticket_ = 1;
    int next_client_ = 0;
    bool stop_ = false;
};

}  // namespace hetal
