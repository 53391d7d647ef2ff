// runtime.cu -- worker pool and tile tuner (see runtime.h).
#include "runtime.h"

#include <algorithm>
#include <cmath>

namespace hetal {

WorkerPool::WorkerPool(const Params &p, int device, int n)
{
    for (int i = 0; i < n; i++) ctxs_.emplace_back(new Context(p, device, nullptr));
}

void WorkerPool::run(size_t njobs, const std::function<void(Context &, size_t)> &fn)
{
    std::atomic<size_t> next{0};
    std::mutex mu;
    std::exception_ptr err;
    std::vector<std::thread> th;
    for (auto &cp : ctxs_) {
        Context *c = cp.get();
        th.emplace_back([&, c] {
            try {
                HETAL_CUDA_CHECK(cudaSetDevice(c->device));
                for (;;) {
                    size_t i = next.fetch_add(1);
                    if (i >= njobs) break;
                    {
                        std::lock_guard<std::mutex> lk(mu);
                        if (err) break;
                    }
                    fn(*c, i);
                }
                c->sync();
            } catch (...) {
                std::lock_guard<std::mutex> lk(mu);
                if (!err) err = std::current_exception();
                cudaStreamSynchronize(c->stream);
            }
        });
    }
    for (auto &t : th) t.join();
    if (err) std::rethrow_exception(err);
}

Counters WorkerPool::counters() const
{
    Counters s;
    for (auto &c : ctxs_) {
        s.cmult += c->cnt.cmult;
        s.mult += c->cnt.mult;
        s.rot += c->cnt.rot;
        s.conj += c->cnt.conj;
        s.keyswitch += c->cnt.keyswitch;
        s.modup_digits += c->cnt.modup_digits;
        s.ntt_limbs += c->cnt.ntt_limbs;
        s.rescale += c->cnt.rescale;
        s.modmul += c->cnt.modmul;
    }
    return s;
}

long long WorkerPool::launches() const
{
    long long n = 0;
    for (auto &c : ctxs_) n += c->launches;
    return n;
}

// ---------------------------------------------------------------------------
void TileTuner::calibrate(Context &c, const EvalKeys &ek)
{
    if (ek.rot.empty()) throw Error(ERR_MISSING_KEY, "tile tuning needs at least one rotation key");
    const int r = ek.rot.begin()->first;
    const Params &p = c.p;
    ks_ms_.assign(p.L, 0.0);
    ks_ms_b_.assign(p.L, 0.0);
    kip_ms_b_.assign(p.L, 0.0);
    cudaEvent_t e0, e1;
    HETAL_CUDA_CHECK(cudaEventCreate(&e0));
    HETAL_CUDA_CHECK(cudaEventCreate(&e1));
    auto time_ms = [&](int reps, const std::function<void()> &fn) {
        fn();   // warm-up (tables, allocator)
        HETAL_CUDA_CHECK(cudaEventRecord(e0, c.stream));
        for (int k = 0; k < reps; k++) fn();
        HETAL_CUDA_CHECK(cudaEventRecord(e1, c.stream));
        HETAL_CUDA_CHECK(cudaEventSynchronize(e1));
        float ms = 0;
        HETAL_CUDA_CHECK(cudaEventElapsedTime(&ms, e0, e1));
        return (double)ms / reps;
    };
    for (int lv = 0; lv < p.L; lv++) {
        for (int which = 0; which < 2; which++) {
            const int B = which ? 32 : 1;
            CtBatch x(&c, B, lv, p.scale);
            HETAL_CUDA_CHECK(cudaMemsetAsync(x.data, 0, sizeof(u64) * B * x.ct_words(), c.stream));
            const double per = time_ms(which ? 2 : 5, [&] { CtBatch y = rotate(c, ek, x.view(), r); });
            if (which) {
                ks_ms_b_[lv] = per / B;
                // a rotation sum of 7 amounts (one key, repeated) against one amount: 6 more key inner products
                const double t7 = time_ms(2, [&] { CtBatch y = rotate_sum(c, ek, x.view(), std::vector<int>(7, r)); });
                const double t1 = time_ms(2, [&] { CtBatch y = rotate_sum(c, ek, x.view(), std::vector<int>(1, r)); });
                kip_ms_b_[lv] = std::max(0.0, (t7 - t1) / 6.0 / B);
            } else {
                ks_ms_[lv] = per;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
}

// time of a batched key switch of `batch` ciphertexts at level lv
double TileTuner::ks(int lv, int batch) const
{
    lv = std::max(0, std::min(lv, (int)ks_ms_.size() - 1));
    double t1 = ks_ms_[lv], tb = ks_ms_b_[lv];
    double marginal = std::max(tb, (32.0 * tb - t1) / 31.0);
    return t1 + (batch - 1) * marginal;
}

// one more summed amount (its key inner product) over `batch` ciphertexts at level lv
double TileTuner::kip(int lv, int batch) const
{
    lv = std::max(0, std::min(lv, (int)kip_ms_b_.size() - 1));
    return batch * kip_ms_b_[lv];
}

// x summed over its rotations by u * unit, u < 2^bits: log-depth rotate-and-add, or radix
// steps (one key switch and 2^b - 2 more key inner products each)
double TileTuner::chain(int lv, int bits, int batch, bool radix) const
{
    if (!radix) return bits * ks(lv, batch);
    double t = 0;
    const int steps = (bits + 2) / 3;
    for (int i = 0; i < steps; i++) {
        const int b = bits / steps + (i < bits % steps ? 1 : 0);
        t += ks(lv, batch) + ((1 << b) - 2) * kip(lv, batch);
    }
    return t;
}

double TileTuner::estimate_ms(const Params &p, int a, int b, int cc, int s0, int flags) const
{
    const int s1 = p.slots() / s0;
    const int m = (a + s0 - 1) / s0, n = (b + s1 - 1) / s1, h = cc / 2;
    const int T = p.L - 1;
    const int lg1 = (int)std::lround(std::log2((double)s1)), lg0 = (int)std::lround(std::log2((double)s0));
    const bool radix = flags & FLAG_RADIX_SUM, shared = flags & FLAG_SHARED_ROT;
    double t = 0;
    // DiagABT: RotUp(B-bar, c/2), the c/2-1 hoisted RotUps (about half the cost each),
    // the c/2 relinearisations per row block, SumCols, Conj
    t += ks(T, n) + 0.5 * (h - 1) * ks(T, n);
    t += m * ks(T, h);
    t += m * (chain(T - 1, lg1, h, radix) + chain(T - 2, lg1, h, radix));
    t += ks(T - 3, m);
    // DiagATB from A at level T-3 (PRotUp branch): RotLeft, Lrot(A_cplx, k), PRotUp,
    // products, SumRows, Conj
    t += (shared ? 1.5 : 2.0) * ks(T - 3, m) + 0.5 * (h - 1) * ks(T - 4, m);
    t += shared ? ks(T - 2, m * n) : ks(T - 3, (h - 1) * m * n);
    t += ks(T - 4, h * n);
    t += chain(T - 5, lg0, h * n, radix);
    t += ks(T - 6, n);
    return t;
}

int TileTuner::choose_s0(const Params &p, int a, int b, int cc) const
{
    int best = -1;
    double bt = 0;
    for (int s0 = cc; s0 <= p.slots() / cc; s0 *= 2) {
        double t = estimate_ms(p, a, b, cc, s0);
        if (best < 0 || t < bt) {
            best = s0;
            bt = t;
        }
    }
    if (best < 0) throw Error(ERR_SHAPE, "no block shape satisfies c <= min(s0, s1)");
    return best;
}

std::pair<int, int> TileTuner::choose(const Params &p, int a, int b, int cc) const
{
    std::pair<int, int> best(-1, 0);
    double bt = 0;
    for (int s0 = cc; s0 <= p.slots() / cc; s0 *= 2)
        for (int extra : {0, (int)FLAG_RADIX_SUM, (int)FLAG_SHARED_ROT, (int)(FLAG_RADIX_SUM | FLAG_SHARED_ROT)}) {
            const int f = FLAG_HOIST | FLAG_LAZY_RELIN | extra;
            double t = estimate_ms(p, a, b, cc, s0, f);
            if (best.first < 0 || t < bt) {
                best = {s0, f};
                bt = t;
            }
        }
    if (best.first < 0) throw Error(ERR_SHAPE, "no block shape satisfies c <= min(s0, s1)");
    return best;
}

}  // namespace hetal
