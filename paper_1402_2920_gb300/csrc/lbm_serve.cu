// Continuous-batching serving loop over the public entry points.
//
// Requests arrive over time.  Each is admitted as soon as it has arrived, a slot is free
// and its device footprint fits the memory budget (first come, first served: a request
// that does not fit yet holds back the ones behind it).  Every admitted simulation keeps
// its populations resident and advances in chunks of steps, and the host loop only issues
// chunks, polls their completion events, retires finished requests (fields back to the
// caller's host buffers) and admits new ones in the slots and memory they free.
//
// Two ways of advancing the resident simulations:
//   batched   the simulations of one kernel combination (lattice, storage, u-solve precision,
//             gamma = 0 or not) and size class form a batch whose chunk is one graph launch per step: each
//             stage of the step is one persistent launch over the tiles of every simulation in
//             the batch (lbm_batch.h).  A batch takes its next chunk once the previous one is
//             done; waiting requests of that combination join in between.  Batches of
//             different combinations run on their own streams.
//   streams   each simulation on its own stream, its chunk that many launches of its own step
//             graph; the kernels of all of them overlap on the device.
#include <algorithm>
#include <chrono>
#include <cstdint>
#include <deque>
#include <thread>
#include <vector>

#include "lbm.h"
#include "lbm_batch.h"

namespace {

struct Slot {
    int req = -1;
    lbm_sim* sim = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    int64_t remaining = 0, in_flight = 0;
    size_t bytes = 0;
};

double seconds_since(std::chrono::steady_clock::time_point t0)
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

// Finish a request: its status, the fields for the caller, the slot and its memory back.
void retire(Slot& sl, const lbm_request* reqs, lbm_request_result* out, int status,
            std::chrono::steady_clock::time_point t0, size_t& used)
{
    const lbm_request& r = reqs[sl.req];
    int rc = status;
    if (rc == LBM_OK) rc = lbm_sync(sl.sim);
    if (rc == LBM_OK && (r.rho_out || r.u_out)) rc = lbm_fields(sl.sim, r.rho_out, r.u_out, 0);
    out[sl.req].status = rc;
    out[sl.req].finish_s = seconds_since(t0);
    lbm_destroy(sl.sim);
    sl.sim = nullptr;
    sl.req = -1;
    used -= sl.bytes;
    sl.bytes = 0;
}

// One stream per simulation.
int serve_streams(const lbm_request* reqs, int n, const lbm_serve_config* cfg, lbm_request_result* out,
                  const std::vector<int>& order, size_t budget)
{
    std::vector<Slot> slots(cfg->max_active);
    int rc = LBM_OK;
    for (Slot& sl : slots) {
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess) {
            rc = LBM_E_CUDA;
            break;
        }
    }
    const auto t0 = std::chrono::steady_clock::now();
    size_t used = 0;
    int next = 0, finished = 0, active = 0;
    while (rc == LBM_OK && finished < n) {
        bool progress = false;
        // admission, first come first served
        while (next < n && active < cfg->max_active) {
            const int k = order[next];
            const lbm_request& r = reqs[k];
            if (r.arrival_s > seconds_since(t0)) break;
            const size_t bytes = lbm_footprint_bytes(r.lattice, r.dims, r.params.storage);
            if (bytes == 0 || bytes > budget) {  // invalid, or can never fit
                out[k].status = bytes == 0 ? LBM_E_INVALID_ARG : LBM_E_OOM;
                out[k].finish_s = seconds_since(t0);
                ++next;
                ++finished;
                progress = true;
                continue;
            }
            if (used + bytes > budget) break;  // wait for memory
            Slot* sl = nullptr;
            for (Slot& s : slots)
                if (s.req < 0) { sl = &s; break; }
            int e = lbm_create(r.lattice, r.dims, &r.eos, &r.params, sl->stream, &sl->sim);
            if (e == LBM_OK) e = lbm_init(sl->sim, r.rho_init, r.u_init, 0);
            ++next;
            progress = true;
            out[k].admit_s = seconds_since(t0);
            out[k].footprint = bytes;
            if (e != LBM_OK) {
                lbm_destroy(sl->sim);
                sl->sim = nullptr;
                out[k].status = e;
                out[k].finish_s = out[k].admit_s;
                ++finished;
                continue;
            }
            sl->req = k;
            sl->remaining = r.steps;
            sl->in_flight = 0;
            sl->bytes = bytes;
            used += bytes;
            ++active;
        }
        // issue the next chunk of every idle simulation; poll the running ones
        for (Slot& sl : slots) {
            if (sl.req < 0) continue;
            if (sl.in_flight == 0) {
                if (sl.remaining == 0) {
                    retire(sl, reqs, out, LBM_OK, t0, used);
                    --active;
                    ++finished;
                    progress = true;
                    continue;
                }
                const int64_t c = std::min<int64_t>(cfg->chunk_steps, sl.remaining);
                int e = lbm_step(sl.sim, c);
                if (e == LBM_OK && cudaEventRecord(sl.done, sl.stream) != cudaSuccess) e = LBM_E_CUDA;
                if (e != LBM_OK) {
                    retire(sl, reqs, out, e, t0, used);
                    --active;
                    ++finished;
                    progress = true;
                    continue;
                }
                sl.in_flight = c;
                progress = true;
            } else {
                const cudaError_t q = cudaEventQuery(sl.done);
                if (q == cudaErrorNotReady) continue;
                progress = true;
                out[sl.req].steps_done += sl.in_flight;
                sl.remaining -= sl.in_flight;
                sl.in_flight = 0;
                if (q != cudaSuccess) (void)cudaGetLastError();
                if (q != cudaSuccess || sl.remaining == 0) {
                    retire(sl, reqs, out, q == cudaSuccess ? LBM_OK : LBM_E_CUDA, t0, used);
                    --active;
                    ++finished;
                }
            }
        }
        if (!progress) {
            if (active == 0 && next < n) {  // idle until the next arrival
                const double wait = reqs[order[next]].arrival_s - seconds_since(t0);
                if (wait > 0) std::this_thread::sleep_for(std::chrono::duration<double>(std::min(wait, 0.01)));
            } else {
                std::this_thread::sleep_for(std::chrono::microseconds(20));
            }
        }
    }
    for (Slot& sl : slots) {  // only after an error: release what is still held
        if (sl.sim) lbm_destroy(sl.sim);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    return rc;
}

// A batch of one kernel combination: its resident requests, their remaining steps, the chunk
// in flight.
struct Family {
    int key = 0;
    lbm::Batch* batch = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    bool in_flight = false;
    int req[lbm::kBatchSlots];
    lbm_sim* sim[lbm::kBatchSlots];
    int64_t remaining[lbm::kBatchSlots];
    int64_t chunk[lbm::kBatchSlots];
    size_t bytes[lbm::kBatchSlots];
    std::deque<int> waiting;  // admitted requests (created, initialised) waiting for the next chunk
    Family()
    {
        for (int k = 0; k < lbm::kBatchSlots; ++k) {
            req[k] = -1;
            sim[k] = nullptr;
            remaining[k] = chunk[k] = 0;
            bytes[k] = 0;
        }
    }
};

// Batched launches per kernel combination.
int serve_batched(const lbm_request* reqs, int n, const lbm_serve_config* cfg, lbm_request_result* out,
                  const std::vector<int>& order, size_t budget)
{
    std::vector<Family> fams;
    std::vector<lbm_sim*> pending(n, nullptr);  // created and initialised, not yet in a batch
    // simulations are created and initialised on this stream while the batches run on theirs
    cudaStream_t admit = nullptr;
    int rc = cudaStreamCreateWithFlags(&admit, cudaStreamNonBlocking) == cudaSuccess ? LBM_OK : LBM_E_CUDA;
    const auto t0 = std::chrono::steady_clock::now();
    size_t used = 0;
    int next = 0, finished = 0, active = 0;
    auto finish = [&](int k, int status, lbm_sim* s, size_t bytes) {
        const lbm_request& r = reqs[k];
        int e = status;
        if (e == LBM_OK) e = lbm_sync(s);
        if (e == LBM_OK && (r.rho_out || r.u_out)) e = lbm_fields(s, r.rho_out, r.u_out, 0);
        out[k].status = e;
        out[k].finish_s = seconds_since(t0);
        lbm_destroy(s);
        used -= bytes;
        --active;
        ++finished;
    };
    while (rc == LBM_OK && finished < n) {
        bool progress = false;
        // admission, first come first served: create and initialise, then wait for the batch
        while (next < n && active < cfg->max_active) {
            const int k = order[next];
            const lbm_request& r = reqs[k];
            if (r.arrival_s > seconds_since(t0)) break;
            const size_t bytes = lbm_footprint_bytes(r.lattice, r.dims, r.params.storage);
            if (bytes == 0 || bytes > budget) {  // invalid, or can never fit
                out[k].status = bytes == 0 ? LBM_E_INVALID_ARG : LBM_E_OOM;
                out[k].finish_s = seconds_since(t0);
                ++next;
                ++finished;
                progress = true;
                continue;
            }
            if (used + bytes > budget) break;  // wait for memory
            const int key = lbm::batch_key(r.lattice, r.dims, r.params);
            Family* f = nullptr;
            for (Family& g : fams)
                if (g.key == key) f = &g;
            int resident = 0;
            if (f) {
                for (int s = 0; s < lbm::kBatchSlots; ++s) resident += f->req[s] >= 0 ? 1 : 0;
                if (resident + int(f->waiting.size()) >= lbm::kBatchSlots) break;  // the batch is full
            }
            lbm_sim* s = nullptr;
            int e = lbm_create(r.lattice, r.dims, &r.eos, &r.params, admit, &s);
            if (e == LBM_OK) e = lbm_init(s, r.rho_init, r.u_init, 0);
            if (e == LBM_OK && !f) {  // the first request of this combination makes its batch
                fams.emplace_back();
                f = &fams.back();
                f->key = key;
                if (cudaStreamCreateWithFlags(&f->stream, cudaStreamNonBlocking) != cudaSuccess ||
                    cudaEventCreateWithFlags(&f->done, cudaEventDisableTiming) != cudaSuccess)
                    e = LBM_E_CUDA;
                if (e == LBM_OK) e = lbm::batch_create(s, f->stream, &f->batch);
            }
            if (e == LBM_OK && cudaStreamSynchronize(admit) != cudaSuccess) e = LBM_E_CUDA;
            ++next;
            progress = true;
            out[k].admit_s = seconds_since(t0);
            out[k].footprint = bytes;
            if (e != LBM_OK) {
                lbm_destroy(s);
                out[k].status = e;
                out[k].finish_s = out[k].admit_s;
                ++finished;
                if (e == LBM_E_CUDA) rc = e;
                continue;
            }
            pending[k] = s;
            f->waiting.push_back(k);
            used += bytes;
            ++active;
        }
        for (Family& f : fams) {
            if (f.in_flight) {
                const cudaError_t q = cudaEventQuery(f.done);
                if (q == cudaErrorNotReady) continue;
                progress = true;
                f.in_flight = false;
                if (q != cudaSuccess) {
                    (void)cudaGetLastError();
                    rc = LBM_E_CUDA;
                    break;
                }
                lbm::batch_account(f.batch, f.chunk);
                for (int s = 0; s < lbm::kBatchSlots; ++s) {
                    if (f.req[s] < 0) continue;
                    out[f.req[s]].steps_done += f.chunk[s];
                    f.remaining[s] -= f.chunk[s];
                    f.chunk[s] = 0;
                }
            }
            // between chunks: retire the finished, seat the waiting, launch the next chunk
            for (int s = 0; s < lbm::kBatchSlots; ++s) {
                if (f.req[s] < 0 || f.remaining[s] > 0) continue;
                lbm::batch_detach(f.batch, s);
                finish(f.req[s], LBM_OK, f.sim[s], f.bytes[s]);
                f.req[s] = -1;
                f.sim[s] = nullptr;
                progress = true;
            }
            for (int s = 0; s < lbm::kBatchSlots && !f.waiting.empty(); ++s) {
                if (f.req[s] >= 0) continue;
                const int k = f.waiting.front();
                f.waiting.pop_front();
                f.req[s] = k;
                f.sim[s] = pending[k];
                pending[k] = nullptr;
                f.remaining[s] = reqs[k].steps;
                f.bytes[s] = out[k].footprint;
                lbm::batch_attach(f.batch, s, f.sim[s]);
                progress = true;
                if (f.remaining[s] == 0) {  // nothing to step: done at once
                    lbm::batch_detach(f.batch, s);
                    finish(k, LBM_OK, f.sim[s], f.bytes[s]);
                    f.req[s] = -1;
                    f.sim[s] = nullptr;
                }
            }
            bool any = false;
            for (int s = 0; s < lbm::kBatchSlots; ++s) {
                f.chunk[s] = f.req[s] >= 0 ? std::min<int64_t>(cfg->chunk_steps, f.remaining[s]) : 0;
                any = any || f.chunk[s] > 0;
            }
            if (!any) continue;
            int e = lbm::batch_launch(f.batch, f.chunk);
            if (e == LBM_OK && cudaEventRecord(f.done, f.stream) != cudaSuccess) e = LBM_E_CUDA;
            if (e != LBM_OK) {
                rc = e;
                break;
            }
            f.in_flight = true;
            progress = true;
        }
        if (!progress) {
            if (active == 0 && next < n) {  // idle until the next arrival
                const double wait = reqs[order[next]].arrival_s - seconds_since(t0);
                if (wait > 0) std::this_thread::sleep_for(std::chrono::duration<double>(std::min(wait, 0.01)));
            } else {
                std::this_thread::sleep_for(std::chrono::microseconds(20));
            }
        }
    }
    for (Family& f : fams) {  // release everything (only an error leaves simulations behind)
        if (f.stream) cudaStreamSynchronize(f.stream);
        for (int s = 0; s < lbm::kBatchSlots; ++s)
            if (f.sim[s]) lbm_destroy(f.sim[s]);
        lbm::batch_destroy(f.batch);
        if (f.done) cudaEventDestroy(f.done);
        if (f.stream) cudaStreamDestroy(f.stream);
    }
    for (lbm_sim* s : pending)
        if (s) lbm_destroy(s);
    if (admit) cudaStreamDestroy(admit);
    return rc;
}

}  // namespace

extern "C" int lbm_serve(const lbm_request* reqs, int n, const lbm_serve_config* cfg, lbm_request_result* out)
{
    if (n < 0 || (n > 0 && (!reqs || !out)) || !cfg) return LBM_E_INVALID_ARG;
    if (cfg->max_active < 1 || cfg->chunk_steps < 1) return LBM_E_INVALID_ARG;
    if (n == 0) return LBM_OK;
    for (int k = 0; k < n; ++k) {
        if (!reqs[k].rho_init || reqs[k].steps < 0 || !(reqs[k].arrival_s >= 0.0)) return LBM_E_INVALID_ARG;
        out[k].admit_s = -1.0;
        out[k].finish_s = -1.0;
        out[k].status = LBM_E_INVALID_ARG;
        out[k].steps_done = 0;
        out[k].footprint = 0;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LBM_E_CUDA;
    size_t budget = cfg->memory_budget;
    if (budget == 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return LBM_E_CUDA;
        budget = fr / 10 * 9;
    }
    // freed simulation memory stays in the stream-ordered pool for the next admissions
    cudaMemPool_t pool = nullptr;
    uint64_t old_threshold = 0;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &old_threshold);
        uint64_t keep = budget;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    std::vector<int> order(n);
    for (int k = 0; k < n; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return reqs[a].arrival_s < reqs[b].arrival_s; });
    const int rc = cfg->batched ? serve_batched(reqs, n, cfg, out, order, budget)
                                : serve_streams(reqs, n, cfg, out, order, budget);
    if (pool) cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &old_threshold);
    return rc;
}
