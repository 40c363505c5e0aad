// Continuous-batching serving loop over the public entry points.
//
// Requests arrive over time.  Each is admitted as soon as it has arrived, a slot is free
// and its device footprint fits the memory budget (first come, first served: a request
// that does not fit yet holds back the ones behind it).  Every admitted simulation keeps
// its populations resident and advances on its own stream in chunks of graph-launched
// steps, so the work of all of them overlaps on the device.  The host loop only issues
// chunks, polls their completion events, retires finished requests (fields back to the
// caller's host buffers) and admits new ones in the slots and memory they free.
#include <algorithm>
#include <chrono>
#include <cstdint>
#include <thread>
#include <vector>

#include "lbm.h"

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
    if (pool) cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &old_threshold);
    return rc;
}
