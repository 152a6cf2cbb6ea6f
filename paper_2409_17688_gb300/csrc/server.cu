// Serving: a continuous-batching gamma_2(P_n x C_m) server (Theorem 2).
//
// For every path order it serves, the server keeps powers of A(D_n)
// resident on the device: the "baby steps" A^1..A^B (from the sparse chain)
// and, transposed, the "giant steps" A^{tB}, t = 1..T (dense products
// A^{tB} = A^{(t-1)B} (x) A^B).  For m <= B the answer is the min-diagonal
// of A^m, kept on the host from the chain.  Any larger m <= B(T+1) splits as
// m = x + tB with x in [1, B], and gamma_2 = min_i (A^x (x) A^{tB})_ii =
// min_{i,l} A^x_il + (A^{tB})^T_il: one streaming pass over two resident
// matrices (a min of elementwise sums, 16-bit pairs, 16-byte loads).
//
// Requests enter a queue (mp_server_submit, any host thread).  A worker
// thread drains it continuously: queries whose n is resident join the next
// batch, which runs as one launch of the batched min-trace kernel on the
// compute stream (at most two batches in flight, so a new batch is formed
// while the previous one runs).  A query for a path order that is not
// resident triggers its admission: the footprint (B + T - 1) N^2 int16 is
// checked against the device-memory budget, least recently used path orders
// with no queries in flight are evicted until it fits, and a builder thread
// computes the powers on its own stream, so building overlaps the batches
// of other path orders.  Queries that arrive meanwhile wait for it.
// Footprints larger than the whole budget are refused with MP_ENOMEM; a full
// ticket table is refused with MP_EBUSY.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "mp_internal.cuh"

extern "C" int mp_transfer_power_sequence(int n, int k_max, int16_t *powers_opt,
                                          int32_t *gdiag_opt, void *stream);

namespace mp {

namespace {

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct TraceJob {
    const int16_t *X;   // A^x, representative rows first
    const int16_t *YT;  // (A^{tB})^T, rows in the same order
    int64_t count;      // representative rows x N
    int64_t cta0;       // first CTA of this job
};

constexpr int kTraceThreads = 256;
constexpr int64_t kTraceSpan = (int64_t)kTraceThreads * 8 * 16;  // entries per CTA

// min over e of X[e] + YT[e] for every job; each CTA takes one contiguous
// span of one job (both slots start on 16-byte boundaries, spans are
// multiples of 8 entries), folds 16-bit pairs with __viaddmin_u16x2 and
// issues one atomicMin.
__global__ void __launch_bounds__(kTraceThreads)
trace_stream_kernel(const TraceJob *__restrict__ jobs, int njobs, int32_t *__restrict__ out) {
    int lo = 0, hi = njobs - 1;
    const int64_t b = blockIdx.x;
    while (lo < hi) {  // last job with cta0 <= b
        const int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].cta0 <= b) lo = mid;
        else hi = mid - 1;
    }
    const TraceJob j = jobs[lo];
    const int64_t start = (b - j.cta0) * kTraceSpan;
    const int64_t end = min(j.count, start + kTraceSpan);
    const int64_t vend = start + ((end - start) & ~(int64_t)7);
    uint32_t acc = 0xFFFFFFFFu;
    for (int64_t e = start + 8 * (int64_t)threadIdx.x; e < vend; e += 8 * kTraceThreads) {
        const uint4 x = __ldg(reinterpret_cast<const uint4 *>(j.X + e));
        const uint4 y = __ldg(reinterpret_cast<const uint4 *>(j.YT + e));
        acc = __viaddmin_u16x2(x.x, y.x, acc);
        acc = __viaddmin_u16x2(x.y, y.y, acc);
        acc = __viaddmin_u16x2(x.z, y.z, acc);
        acc = __viaddmin_u16x2(x.w, y.w, acc);
    }
    int32_t v = (int32_t)min(acc & 0xFFFFu, acc >> 16);
    for (int64_t e = vend + threadIdx.x; e < end; e += kTraceThreads)
        v = min(v, (int32_t)(uint16_t)j.X[e] + (int32_t)(uint16_t)j.YT[e]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
    __shared__ int32_t wmin[kTraceThreads / 32];
    if ((threadIdx.x & 31) == 0) wmin[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kTraceThreads / 32; ++w) v = min(v, wmin[w]);
        v = min(v, (int32_t)kInf16);
        if (v < (int32_t)kInf16) atomicMin(&out[lo], v);
    }
}

// out[c][r] = in[r][c] for an N x N matrix (both with leading dimension ld_in / N).
__global__ void transpose_kernel(const int16_t *__restrict__ in, int64_t ld_in,
                                 int16_t *__restrict__ out, int64_t N) {
    __shared__ int16_t t[32][33];
    const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t rr = r0 + r, cc = c0 + threadIdx.x;
        if (rr < N && cc < N) t[r][threadIdx.x] = in[rr * ld_in + cc];
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t oc = c0 + r, orow = r0 + threadIdx.x;  // out[oc][orow] = in[orow][oc]
        if (oc < N && orow < N) out[oc * N + orow] = t[threadIdx.x][r];
    }
}

// out row r = in row rows[r] (N entries each, both packed); one CTA per row.
__global__ void row_gather_kernel(const int16_t *__restrict__ in, const int32_t *__restrict__ rows,
                                  int64_t N, int16_t *__restrict__ out) {
    const int16_t *src = in + (int64_t)rows[blockIdx.x] * N;
    int16_t *dst = out + (int64_t)blockIdx.x * N;
    for (int64_t c = threadIdx.x; c < N; c += blockDim.x) dst[c] = src[c];
}

__global__ void fill_inf_kernel(int32_t *p, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        p[i] = (int32_t)kInf16;
}

enum SlotState : int { kFree = 0, kQueued = 1, kDone = 2, kFailed = 3, kCancelled = 4 };

struct Slot {
    std::atomic<int> state{kFree};
    int64_t value = 0;
    int err = 0;
    int n = 0;
    int64_t m = 0;
    double t_submit = 0, t_done = 0;
};

struct Query {
    uint64_t ticket;
    int n;
    int64_t m;
};

enum NStatus { kAbsent = 0, kBuilding = 1, kResident = 2 };

struct PathState {
    int n = 0;
    int64_t N = 0;
    int status = kAbsent;
    size_t bytes = 0;
    int16_t *powers = nullptr;  // B + T slots of `slot` entries: A^1..A^B, then (A^{tB})^T
    size_t slot = 0;            // N*N rounded up to 8 entries (16-byte aligned slots)
    int64_t nrep = 0;           // rows a trace reads: one word of every mirror pair
    std::vector<int32_t> diag;  // min diag A^m, m = 1..B
    std::atomic<int> built{0};  // set by the builder thread (1 ok, -1 failed)
    int build_err = 0;
    std::thread builder;
    uint64_t last_use = 0;
    int inflight = 0;
    std::deque<Query> waiting;
};

struct Batch {
    std::vector<Query> qs;
    int64_t ctas = 0;
    std::vector<std::pair<int, int>> uses;  // path orders touched (n, count)
    int32_t *d_out = nullptr;
    int32_t *h_out = nullptr;
    TraceJob *d_jobs = nullptr;
    TraceJob *h_jobs = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    nvtxRangeId_t range = 0;  // NVTX range of the batch in flight
};

}  // namespace

}  // namespace mp

struct mp_server {
    // configuration
    int device = 0;
    size_t budget = 0;
    int max_batch = 0;
    int64_t max_m = 0;
    int B = 0, T = 0;
    int sms = 0;
    // tickets
    std::vector<mp::Slot> slots;
    std::atomic<uint64_t> next_ticket{0};
    // queue
    std::mutex mu;
    std::condition_variable cv;
    std::deque<mp::Query> queue;
    bool stop = false;
    // worker state
    std::thread worker;
    cudaStream_t compute = nullptr;
    std::map<int, std::unique_ptr<mp::PathState>> paths;
    size_t used = 0;
    uint64_t clock = 0;
    mp::Batch batches[2];
    std::deque<mp::Query> deferred;
    // statistics
    std::atomic<uint64_t> stat_completed{0}, stat_failed{0}, stat_batches{0}, stat_builds{0},
        stat_evictions{0}, stat_cancelled{0};
    std::atomic<uint64_t> stat_resident_bytes{0};
};

namespace mp {

namespace {

size_t slot_of(int64_t N) { return ((size_t)N * (size_t)N + 7) & ~(size_t)7; }

size_t footprint(const mp_server *sv, int64_t N) {
    return (size_t)(sv->B + sv->T) * slot_of(N) * 2;
}

int64_t words_count(int n) {
    std::vector<uint32_t> w;
    enumerate_words(n, &w);
    return (int64_t)w.size();
}

// Builder thread body, on a private stream: baby steps by the sparse chain
// (with their min-diagonals), giant steps by dense products in padded
// scratch, each stored transposed.  Last, the rows of every slot are put in
// one order that lists first one word of every mirror pair {q, R q} (R reads
// a word backwards).  R is an automorphism of A(D_n), so P_x[R i][R l] =
// P_x[i][l] for every power, and the trace term P_x[i][l] + P_y[l][i] of the
// pair (i, l) equals that of (R i, R l): the minimum over the representative
// rows and all columns is the minimum over all of them, and a trace reads
// about half of each slot.
void build_path(mp_server *sv, PathState *ps) {
    NvtxScope nv("mp_server build n=%d", ps->n);
    cudaSetDevice(sv->device);
    cudaStream_t s = nullptr;
    int rc = MP_OK;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) rc = MP_ECUDA;
    const int64_t N = ps->N;
    const int64_t ld = (N + 7) & ~(int64_t)7;  // padded rows: 16-byte vector loads in the products
    ps->slot = slot_of(N);
    int16_t *tmp = nullptr;
    int32_t *gd = nullptr;
    if (rc == MP_OK && cudaMallocAsync((void **)&ps->powers, footprint(sv, N), s) != cudaSuccess) {
        ps->powers = nullptr;
        rc = MP_ENOMEM;
    }
    if (rc == MP_OK && (cudaMallocAsync((void **)&tmp, (size_t)3 * N * ld * 2, s) != cudaSuccess ||
                        cudaMallocAsync((void **)&gd, sizeof(int32_t) * (size_t)sv->B, s) != cudaSuccess))
        rc = MP_ENOMEM;
    if (rc == MP_OK) rc = transfer_powers_strided(ps->n, sv->B, ps->powers, ps->slot, gd, s);
    ps->diag.assign((size_t)sv->B, 0);
    if (rc == MP_OK && cudaMemcpyAsync(ps->diag.data(), gd, sizeof(int32_t) * (size_t)sv->B,
                                       cudaMemcpyDeviceToHost, s) != cudaSuccess)
        rc = MP_ECUDA;
    int16_t *giant = ps->powers + (size_t)sv->B * ps->slot;
    int16_t *AB = tmp, *cur = tmp + (size_t)N * ld, *nxt = tmp + (size_t)2 * N * ld;
    const dim3 tgrid((unsigned)((N + 31) / 32), (unsigned)((N + 31) / 32)), tblock(32, 8);
    if (rc == MP_OK &&
        cudaMemcpy2DAsync(AB, (size_t)ld * 2, ps->powers + (size_t)(sv->B - 1) * ps->slot,
                          (size_t)N * 2, (size_t)N * 2, (size_t)N, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        rc = MP_ECUDA;
    if (rc == MP_OK) {
        transpose_kernel<<<tgrid, tblock, 0, s>>>(AB, ld, giant, N);  // t = 1
        if (cudaGetLastError() != cudaSuccess) rc = MP_ECUDA;
    }
    const int16_t *prev = AB;
    int16_t *sbuf[2] = {cur, nxt};
    for (int t = 2; rc == MP_OK && t <= sv->T; ++t) {
        int16_t *dst = sbuf[t & 1];
        rc = dense_minplus(prev, AB, dst, N, N, N, ld, ld, ld, MP_I16, nullptr, s);
        if (rc != MP_OK) break;
        transpose_kernel<<<tgrid, tblock, 0, s>>>(dst, ld, giant + (size_t)(t - 1) * ps->slot, N);
        if (cudaGetLastError() != cudaSuccess) rc = MP_ECUDA;
        prev = dst;
    }
    // representative rows (i <= R i) first; the rows after them are never read
    int32_t *d_rows = nullptr;
    std::vector<int32_t> reps;
    if (rc == MP_OK) {
        std::vector<uint32_t> w;
        enumerate_words(ps->n, &w);
        std::vector<int64_t> partner;
        rc = mirror_words(ps->n, w, &partner);
        for (int64_t i = 0; rc == MP_OK && i < N; ++i)
            if (i <= partner[(size_t)i]) reps.push_back((int32_t)i);
    }
    if (rc == MP_OK && cudaMallocAsync((void **)&d_rows, sizeof(int32_t) * reps.size(), s) != cudaSuccess)
        rc = MP_ENOMEM;
    if (rc == MP_OK && cudaMemcpyAsync(d_rows, reps.data(), sizeof(int32_t) * reps.size(),
                                       cudaMemcpyHostToDevice, s) != cudaSuccess)
        rc = MP_ECUDA;
    const int64_t nrep = (int64_t)reps.size();
    for (int k = 0; rc == MP_OK && k < sv->B + sv->T; ++k) {
        int16_t *slot = ps->powers + (size_t)k * ps->slot;
        row_gather_kernel<<<(unsigned)nrep, 256, 0, s>>>(slot, d_rows, N, tmp);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(slot, tmp, sizeof(int16_t) * (size_t)(nrep * N), cudaMemcpyDeviceToDevice,
                            s) != cudaSuccess)
            rc = MP_ECUDA;
    }
    ps->nrep = nrep;
    if (d_rows) cudaFreeAsync(d_rows, s);
    if (tmp) cudaFreeAsync(tmp, s);
    if (gd) cudaFreeAsync(gd, s);
    if (s) {
        if (cudaStreamSynchronize(s) != cudaSuccess && rc == MP_OK) rc = MP_ECUDA;
        cudaStreamDestroy(s);
    }
    ps->build_err = rc;
    ps->built.store(rc == MP_OK ? 1 : -1, std::memory_order_release);
    sv->cv.notify_all();
}

void finish(mp_server *sv, uint64_t ticket, int err, int64_t value) {
    Slot &sl = sv->slots[ticket];
    sl.value = value;
    sl.err = err;
    sl.t_done = now_s();
    int expect = kQueued;
    if (sl.state.compare_exchange_strong(expect, err == MP_OK ? kDone : kFailed)) {
        if (err == MP_OK) sv->stat_completed++;
        else sv->stat_failed++;
    }
}

// A query of a resident path order: m <= B is answered from the host table
// of min-diagonals, larger m goes to the next batch.
void dispatch_resident(mp_server *sv, PathState *ps, const Query &q, std::vector<Query> &ready) {
    if (q.m <= sv->B) {
        ps->last_use = ++sv->clock;
        finish(sv, q.ticket, MP_OK, ps->diag[(size_t)q.m - 1]);
    } else {
        ready.push_back(q);
    }
}

// Route incoming queries: resident -> ready; building -> waiting; absent ->
// admission (evict, start a builder) or refusal.
void route(mp_server *sv, const Query &q, std::vector<Query> &ready) {
    auto it = sv->paths.find(q.n);
    if (it != sv->paths.end() && it->second->status == kResident) {
        dispatch_resident(sv, it->second.get(), q, ready);
        return;
    }
    if (it != sv->paths.end() && it->second->status == kBuilding) {
        it->second->waiting.push_back(q);
        return;
    }
    const int64_t N = words_count(q.n);
    const size_t need = footprint(sv, N);
    if (need > sv->budget) {
        set_error(MP_ENOMEM, "path order %d needs %zu bytes, budget %zu", q.n, need, sv->budget);
        finish(sv, q.ticket, MP_ENOMEM, 0);
        return;
    }
    // evict least recently used idle path orders until the new one fits
    while (sv->used + need > sv->budget) {
        PathState *victim = nullptr;
        for (auto &kv : sv->paths) {
            PathState *p = kv.second.get();
            if (p->status == kResident && p->inflight == 0 && p->waiting.empty() &&
                (!victim || p->last_use < victim->last_use))
                victim = p;
        }
        if (!victim) break;
        cudaFreeAsync(victim->powers, sv->compute);
        victim->powers = nullptr;
        victim->status = kAbsent;
        sv->used -= victim->bytes;
        victim->bytes = 0;
        sv->stat_evictions++;
    }
    if (sv->used + need > sv->budget) {
        sv->deferred.push_back(q);  // admitted once memory frees up
        return;
    }
    auto &ptr = sv->paths[q.n];
    if (!ptr) ptr.reset(new PathState());
    PathState *ps = ptr.get();
    if (ps->builder.joinable()) ps->builder.join();
    ps->n = q.n;
    ps->N = N;
    ps->status = kBuilding;
    ps->bytes = need;
    ps->built.store(0);
    sv->used += need;
    sv->stat_builds++;
    ps->waiting.push_back(q);
    ps->builder = std::thread(build_path, sv, ps);
}

int launch_batch(mp_server *sv, Batch &b, std::vector<Query> &ready) {
    const int cnt = (int)std::min<size_t>(ready.size(), (size_t)sv->max_batch);
    // the batch's lifetime, from launch to completion (ended in complete_batch)
    {
        char name[64];
        snprintf(name, sizeof name, "mp_server batch %llu (%d queries)",
                 (unsigned long long)sv->stat_batches, cnt);
        b.range = nvtxRangeStartA(name);
    }
    b.qs.assign(ready.begin(), ready.begin() + cnt);
    ready.erase(ready.begin(), ready.begin() + cnt);
    std::map<int, int> use;
    int64_t ctas = 0;
    for (int i = 0; i < cnt; ++i) {
        const Query &q = b.qs[i];
        PathState *ps = sv->paths[q.n].get();
        const int64_t t = (q.m - 1) / sv->B;  // m = x + tB, x in [1, B], t in [1, T]
        const int64_t x = q.m - t * sv->B;
        TraceJob &j = b.h_jobs[i];
        j.X = ps->powers + (size_t)(x - 1) * ps->slot;
        j.YT = ps->powers + (size_t)(sv->B + t - 1) * ps->slot;
        j.count = ps->nrep * ps->N;
        j.cta0 = ctas;
        ctas += (j.count + kTraceSpan - 1) / kTraceSpan;
        ps->inflight++;
        ps->last_use = ++sv->clock;
        use[q.n]++;
    }
    b.uses.assign(use.begin(), use.end());
    b.ctas = ctas;
    MP_CUDA_TRY(cudaMemcpyAsync(b.d_jobs, b.h_jobs, sizeof(TraceJob) * (size_t)cnt,
                                cudaMemcpyHostToDevice, sv->compute));
    fill_inf_kernel<<<(cnt + 255) / 256, 256, 0, sv->compute>>>(b.d_out, cnt);
    trace_stream_kernel<<<(unsigned)ctas, kTraceThreads, 0, sv->compute>>>(b.d_jobs, cnt, b.d_out);
    MP_CUDA_TRY(cudaGetLastError());
    MP_CUDA_TRY(cudaMemcpyAsync(b.h_out, b.d_out, sizeof(int32_t) * (size_t)cnt,
                                cudaMemcpyDeviceToHost, sv->compute));
    MP_CUDA_TRY(cudaEventRecord(b.done, sv->compute));
    b.busy = true;
    sv->stat_batches++;
    return MP_OK;
}

void complete_batch(mp_server *sv, Batch &b) {
    nvtxRangeEnd(b.range);
    for (size_t i = 0; i < b.qs.size(); ++i) finish(sv, b.qs[i].ticket, MP_OK, b.h_out[i]);
    for (auto &u : b.uses) sv->paths[u.first]->inflight -= u.second;
    b.qs.clear();
    b.busy = false;
}

void worker_main(mp_server *sv) {
    cudaSetDevice(sv->device);
    std::vector<Query> ready;
    while (true) {
        std::deque<Query> incoming;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            const bool idle = sv->queue.empty() && ready.empty() && !sv->batches[0].busy &&
                              !sv->batches[1].busy;
            if (idle && !sv->stop) {
                bool building = false;
                for (auto &kv : sv->paths) building |= kv.second->status == kBuilding;
                sv->cv.wait_for(lk, std::chrono::microseconds(building ? 100 : 2000));
            }
            if (sv->stop) break;
            incoming.swap(sv->queue);
        }
        // builds that finished: their waiting queries become ready
        for (auto &kv : sv->paths) {
            PathState *ps = kv.second.get();
            if (ps->status != kBuilding) continue;
            const int st = ps->built.load(std::memory_order_acquire);
            if (st == 0) continue;
            if (ps->builder.joinable()) ps->builder.join();
            if (st > 0) {
                ps->status = kResident;
                for (auto &q : ps->waiting) dispatch_resident(sv, ps, q, ready);
            } else {
                for (auto &q : ps->waiting) finish(sv, q.ticket, ps->build_err, 0);
                if (ps->powers) cudaFreeAsync(ps->powers, sv->compute);
                ps->powers = nullptr;
                ps->status = kAbsent;
                sv->used -= ps->bytes;
                ps->bytes = 0;
            }
            ps->waiting.clear();
        }
        // deferred admissions retry once memory may have freed up
        if (!sv->deferred.empty()) {
            std::deque<Query> d;
            d.swap(sv->deferred);
            for (auto &q : d) incoming.push_back(q);
        }
        for (auto &q : incoming) {
            if (sv->slots[q.ticket].state.load() == kCancelled) continue;
            route(sv, q, ready);
        }
        // drop cancelled queries before they are batched
        ready.erase(std::remove_if(ready.begin(), ready.end(),
                                   [&](const Query &q) {
                                       return sv->slots[q.ticket].state.load() == kCancelled;
                                   }),
                    ready.end());
        // completed batches
        for (auto &b : sv->batches)
            if (b.busy && cudaEventQuery(b.done) == cudaSuccess) complete_batch(sv, b);
        // new batches while a slot is free
        for (auto &b : sv->batches)
            if (!b.busy && !ready.empty()) {
                if (launch_batch(sv, b, ready) != MP_OK) {
                    for (auto &q : b.qs) finish(sv, q.ticket, MP_ECUDA, 0);
                    b.qs.clear();
                }
            }
        sv->stat_resident_bytes = sv->used;
        if (!sv->batches[0].busy && !sv->batches[1].busy && ready.empty()) continue;
        std::this_thread::yield();
    }
    // shutdown: let in-flight work finish
    for (auto &b : sv->batches)
        if (b.busy) {
            cudaEventSynchronize(b.done);
            complete_batch(sv, b);
        }
}

}  // namespace

}  // namespace mp

using namespace mp;

extern "C" {

int mp_server_create(size_t hbm_budget, int max_batch, int64_t max_m, int64_t max_tickets,
                     mp_server **out) {
    if (!out || max_batch < 1 || max_m < 3 || max_tickets < 1)
        return set_error(MP_EINVAL, "bad server parameters");
    *out = nullptr;
    auto sv = std::make_unique<mp_server>();
    MP_CUDA_TRY(cudaGetDevice(&sv->device));
    DeviceInfo di;
    MP_TRY(device_info(&di));
    sv->sms = di.sms;
    sv->budget = hbm_budget;
    sv->max_batch = max_batch;
    sv->max_m = max_m;
    int B = 1;
    while ((int64_t)B * B < max_m) ++B;
    sv->B = B;
    sv->T = (int)std::max<int64_t>(2, (max_m + B - 1) / B);
    sv->slots = std::vector<Slot>((size_t)max_tickets);
    MP_CUDA_TRY(cudaStreamCreateWithFlags(&sv->compute, cudaStreamNonBlocking));
    for (auto &b : sv->batches) {
        MP_CUDA_TRY(cudaMalloc(&b.d_out, sizeof(int32_t) * (size_t)max_batch));
        MP_CUDA_TRY(cudaMalloc(&b.d_jobs, sizeof(TraceJob) * (size_t)max_batch));
        MP_CUDA_TRY(cudaMallocHost(&b.h_out, sizeof(int32_t) * (size_t)max_batch));
        MP_CUDA_TRY(cudaMallocHost(&b.h_jobs, sizeof(TraceJob) * (size_t)max_batch));
        MP_CUDA_TRY(cudaEventCreateWithFlags(&b.done, cudaEventDisableTiming));
    }
    mp_server *raw = sv.release();
    raw->worker = std::thread(worker_main, raw);
    *out = raw;
    return MP_OK;
}

int mp_server_submit(mp_server *sv, int n, int64_t m, uint64_t *ticket) {
    if (!sv || !ticket) return set_error(MP_EINVAL, "NULL server or ticket");
    if (n < 1 || n > MP_MAX_PATH_ORDER || m < 3 || m > sv->max_m)
        return set_error(MP_EINVAL, "query (n = %d, m = %lld) outside n in [1, %d], m in [3, %lld]",
                         n, (long long)m, MP_MAX_PATH_ORDER, (long long)sv->max_m);
    if (m * (int64_t)n >= (int64_t)kInf16)
        return set_error(MP_ERANGE, "m * n = %lld reaches the int16 INF code", (long long)(m * n));
    const uint64_t t = sv->next_ticket.fetch_add(1);
    if (t >= sv->slots.size()) {
        sv->next_ticket.fetch_sub(1);
        return set_error(MP_EBUSY, "ticket table full (%zu)", sv->slots.size());
    }
    Slot &sl = sv->slots[t];
    sl.n = n;
    sl.m = m;
    sl.t_submit = now_s();
    sl.state.store(kQueued);
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->queue.push_back({t, n, m});
    }
    sv->cv.notify_one();
    *ticket = t;
    return MP_OK;
}

int mp_server_replay(mp_server *sv, const int32_t *n, const int64_t *m, const double *t_offsets,
                     int64_t count, uint64_t *tickets) {
    if (!sv || !n || !m || !tickets || count < 0) return set_error(MP_EINVAL, "bad replay arguments");
    const double base = now_s();
    for (int64_t i = 0; i < count; ++i) {
        if (t_offsets) {
            const double target = base + t_offsets[i];
            while (now_s() < target) {
            }
        }
        const int rc = mp_server_submit(sv, n[i], m[i], &tickets[i]);
        if (rc != MP_OK) return rc;
    }
    return MP_OK;
}

int mp_server_poll(mp_server *sv, uint64_t ticket, int64_t *gamma2) {
    if (!sv || ticket >= sv->next_ticket.load()) return set_error(MP_EINVAL, "unknown ticket");
    Slot &sl = sv->slots[ticket];
    const int st = sl.state.load(std::memory_order_acquire);
    if (st == kQueued) return MP_ENOTREADY;
    if (st == kCancelled) return set_error(MP_EINVAL, "ticket %llu was cancelled", (unsigned long long)ticket);
    if (st == kFailed) return set_error(sl.err, "query failed");
    if (gamma2) *gamma2 = sl.value;
    return MP_OK;
}

int mp_server_cancel(mp_server *sv, uint64_t ticket) {
    if (!sv || ticket >= sv->next_ticket.load()) return set_error(MP_EINVAL, "unknown ticket");
    int expect = kQueued;
    if (sv->slots[ticket].state.compare_exchange_strong(expect, kCancelled)) {
        sv->stat_cancelled++;
        return MP_OK;
    }
    return set_error(MP_EBUSY, "ticket %llu already finished", (unsigned long long)ticket);
}

int mp_server_latency(mp_server *sv, uint64_t ticket, double *submit_s, double *done_s) {
    if (!sv || ticket >= sv->next_ticket.load()) return set_error(MP_EINVAL, "unknown ticket");
    Slot &sl = sv->slots[ticket];
    const int st = sl.state.load(std::memory_order_acquire);
    if (st != kDone && st != kFailed) return MP_ENOTREADY;
    if (submit_s) *submit_s = sl.t_submit;
    if (done_s) *done_s = sl.t_done;
    return MP_OK;
}

int mp_server_stats(mp_server *sv, int64_t *out) {
    if (!sv || !out) return set_error(MP_EINVAL, "NULL argument");
    out[0] = (int64_t)sv->next_ticket.load();
    out[1] = (int64_t)sv->stat_completed.load();
    out[2] = (int64_t)sv->stat_failed.load();
    out[3] = (int64_t)sv->stat_cancelled.load();
    out[4] = (int64_t)sv->stat_batches.load();
    out[5] = (int64_t)sv->stat_builds.load();
    out[6] = (int64_t)sv->stat_evictions.load();
    out[7] = (int64_t)sv->stat_resident_bytes.load();
    return MP_OK;
}

int mp_server_destroy(mp_server *sv) {
    if (!sv) return MP_OK;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv.notify_all();
    if (sv->worker.joinable()) sv->worker.join();
    for (auto &kv : sv->paths) {
        PathState *ps = kv.second.get();
        if (ps->builder.joinable()) ps->builder.join();
        if (ps->powers) cudaFreeAsync(ps->powers, sv->compute);
    }
    cudaStreamSynchronize(sv->compute);
    for (auto &b : sv->batches) {
        cudaFree(b.d_out);
        cudaFree(b.d_jobs);
        cudaFreeHost(b.h_out);
        cudaFreeHost(b.h_jobs);
        cudaEventDestroy(b.done);
    }
    cudaStreamDestroy(sv->compute);
    delete sv;
    return MP_OK;
}

}  // extern "C"
