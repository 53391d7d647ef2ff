// server.cu -- continuous-batching request loop (see server.h).
#include "server.h"

#include <algorithm>

namespace hetal {

Server::Server(const Params &p, int device, int slots, size_t budget_bytes) : budget_(budget_bytes)
{
    if (slots < 1) throw Error(ERR_INVALID_ARG, "a server needs at least one slot");
    for (int i = 0; i < slots; i++) {
        ctxs_.emplace_back(new Context(p, device, nullptr));
        // each slot's batched operations stay within its share of the budget
        ctxs_.back()->batch_bytes = std::max<size_t>((size_t)256 << 20, budget_bytes / (4 * (size_t)slots));
    }
    assigned_.resize(slots);
    busy_.assign(slots, false);
    for (int i = 0; i < slots; i++) workers_.emplace_back(&Server::worker, this, i);
    sched_ = std::thread(&Server::scheduler, this);
}

Server::~Server()
{
    {
        std::lock_guard<std::mutex> lk(mu_);
        stop_ = true;
    }
    cv_.notify_all();
    work_cv_.notify_all();
    done_cv_.notify_all();
    sched_.join();
    for (auto &t : workers_) t.join();
}

int Server::add_client(const EvalKeys *ek, size_t key_bytes)
{
    std::lock_guard<std::mutex> lk(mu_);
    int id = next_client_++;
    clients_[id] = ek;
    resident_ += key_bytes;
    return id;
}

static size_t mat_bytes(const Mat *m) { return m ? (size_t)m->cts.n * m->cts.ct_words() * sizeof(u64) : 0; }

// Device bytes a request may hold at once: its inputs twice over (dropped or
// rearranged copies) plus two batched operations of its slot.
size_t Server::estimate(const ServerRequest &r) const
{
    return 2 * (mat_bytes(r.a) + mat_bytes(r.b)) + 2 * ctxs_[0]->batch_bytes;
}

uint64_t Server::submit(const ServerRequest &r)
{
    std::lock_guard<std::mutex> lk(mu_);
    if (!clients_.count(r.client)) throw Error(ERR_INVALID_ARG, "unknown client");
    if (!r.a || !r.b) throw Error(ERR_INVALID_ARG, "request without operands");
    const size_t fp = estimate(r), avail = budget_ > resident_ ? budget_ - resident_ : 0;
    if (fp > avail)   // would never be admitted: refused now instead of running into the allocator
        throw Error(ERR_OOM, "request footprint " + std::to_string(fp) + " bytes exceeds the " +
                                 std::to_string(avail) + " bytes the budget leaves beside the resident keys");
    Job j{next_ticket_++, r, fp, std::chrono::steady_clock::now()};
    results_.erase(j.ticket);
    pending_.push_back(j);
    cv_.notify_all();
    return j.ticket;
}

void Server::scheduler()
{
    std::unique_lock<std::mutex> lk(mu_);
    for (;;) {
        cv_.wait(lk, [&] {
            if (stop_) return true;
            if (pending_.empty()) return false;
            bool free_slot = std::find(busy_.begin(), busy_.end(), false) != busy_.end();
            size_t avail = budget_ > resident_ ? budget_ - resident_ : 0;
            bool fits = inflight_ + pending_.front().footprint <= avail;
            return free_slot && fits;
        });
        if (stop_) return;
        // admit in arrival order while slots and memory allow
        while (!pending_.empty()) {
            auto it = std::find(busy_.begin(), busy_.end(), false);
            if (it == busy_.end()) break;
            size_t avail = budget_ > resident_ ? budget_ - resident_ : 0;
            Job &j = pending_.front();
            if (inflight_ + j.footprint > avail) break;
            int slot = (int)(it - busy_.begin());
            busy_[slot] = true;
            inflight_ += j.footprint;
            peak_inflight_ = std::max(peak_inflight_, inflight_);
            assigned_[slot].push_back(j);
            pending_.pop_front();
        }
        work_cv_.notify_all();
    }
}

void Server::worker(int slot)
{
    Context &c = *ctxs_[slot];
    cudaSetDevice(c.device);
    for (;;) {
        Job j;
        {
            std::unique_lock<std::mutex> lk(mu_);
            work_cv_.wait(lk, [&] { return stop_ || !assigned_[slot].empty(); });
            if (stop_ && assigned_[slot].empty()) return;
            j = assigned_[slot].front();
            assigned_[slot].pop_front();
        }
        ServerResult res;
        auto t0 = std::chrono::steady_clock::now();
        res.queue_ms = std::chrono::duration<double, std::milli>(t0 - j.submitted).count();
        res.footprint = j.footprint;
        try {
            const EvalKeys *ek;
            {
                std::lock_guard<std::mutex> lk(mu_);
                ek = clients_.at(j.req.client);
            }
            const ServerRequest &r = j.req;
            res.out = r.kind == 0 ? diag_abt(c, *ek, *r.a, *r.b, r.c, r.t, nullptr, r.flags)
                                  : diag_atb(c, *ek, *r.a, *r.b, r.c, r.t, nullptr, r.flags);
            c.sync();
        } catch (const Error &e) {
            res.status = e.code;
            res.error = e.what();
            if (e.code == ERR_CUDA) cudaGetLastError();
            cudaStreamSynchronize(c.stream);
        } catch (const std::exception &e) {
            res.status = ERR_INVALID_ARG;
            res.error = e.what();
        }
        res.run_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        {
            std::lock_guard<std::mutex> lk(mu_);
            results_[j.ticket] = std::move(res);
            inflight_ -= j.footprint;
            busy_[slot] = false;
            completed_++;
        }
        cv_.notify_all();
        done_cv_.notify_all();
    }
}

bool Server::cancel(uint64_t ticket)
{
    std::lock_guard<std::mutex> lk(mu_);
    for (auto it = pending_.begin(); it != pending_.end(); ++it) {
        if (it->ticket != ticket) continue;
        pending_.erase(it);
        ServerResult res;
        res.status = ERR_CANCELLED;
        res.error = "the request was cancelled before it ran";
        results_[ticket] = std::move(res);
        cv_.notify_all();   // the next queued request may fit now
        done_cv_.notify_all();
        return true;
    }
    return false;
}

bool Server::wait(uint64_t ticket, ServerResult &out)
{
    std::unique_lock<std::mutex> lk(mu_);
    if (ticket == 0 || ticket >= next_ticket_ || taken_.count(ticket)) return false;
    done_cv_.wait(lk, [&] { return stop_ || results_.count(ticket) > 0; });
    auto it = results_.find(ticket);
    if (it == results_.end()) return false;
    out = std::move(it->second);
    results_.erase(it);
    taken_.insert(ticket);
    return true;
}

}  // namespace hetal
