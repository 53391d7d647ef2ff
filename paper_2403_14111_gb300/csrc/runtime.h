// runtime.h -- executors that run many independent encrypted-matmul instances
// (and serving requests) concurrently on one GPU.
#pragma once
#include <atomic>
#include <condition_variable>
#include <deque>
#include <functional>
#include <memory>
#include <mutex>
#include <thread>

#include "matmul.h"

namespace hetal {

// Worker contexts, each with its own CUDA stream, on the same device and
// parameters.  Keys and input ciphertexts made on another context of the same
// device are read directly.  run() hands job i to whichever worker is free, so
// independent instances overlap on the GPU.
class WorkerPool {
  public:
    WorkerPool(const Params &p, int device, int n);
    int size() const { return (int)ctxs_.size(); }
    Context &ctx(int i) { return *ctxs_[i]; }
    void run(size_t njobs, const std::function<void(Context &, size_t)> &fn);
    Counters counters() const;
    long long launches() const;

  private:
    std::vector<std::unique_ptr<Context>> ctxs_;
};

// Tile and variant choice for one DiagABT + DiagATB instance: s0 (s1 = N/2 / s0), a
// power of two with c <= min(s0, s1), and the flags (hoisting and lazy relinearisation
// always; radix sums and shared rotations when they pay), minimising a cost model of
// the instance's key switches whose per-level times are measured on the device
// (calibrate()): a rotation of one ciphertext and, per ciphertext, inside a batch of
// 32; and one more amount of a rotation sum (its key inner product) inside a batch.
class TileTuner {
  public:
    void calibrate(Context &c, const EvalKeys &ek);
    bool calibrated() const { return !ks_ms_.empty(); }
    int choose_s0(const Params &p, int a, int b, int cc) const;
    // best (s0, flags) over the legal tiles and the four variants of FLAG_RADIX_SUM / FLAG_SHARED_ROT
    std::pair<int, int> choose(const Params &p, int a, int b, int cc) const;
    double estimate_ms(const Params &p, int a, int b, int cc, int s0, int flags = 3) const;

  private:
    double ks(int lv, int batch) const;
    double kip(int lv, int batch) const;
    double chain(int lv, int bits, int batch, bool radix) const;
    std::vector<double> ks_ms_;      // one key switch of a single ciphertext, by level
    std::vector<double> ks_ms_b_;    // per ciphertext inside a batch of 32, by level
    std::vector<double> kip_ms_b_;   // one more summed amount, per ciphertext inside a batch of 32, by level
};

}  // namespace hetal
