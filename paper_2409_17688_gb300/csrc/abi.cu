// The exported C ABI (include/minplus.h): argument checks, per-device state
// and the drivers that string the kernels together.
#include <stdarg.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <limits>
#include <map>
#include <memory>
#include <mutex>
#include <tuple>

#include "mp_internal.cuh"
#include "spmm.cuh"

namespace mp {

int dpx_peak(int variant, int64_t iters, double *ops_per_s);
int powers_save(const char *path, int n, int k0, int64_t count, const int16_t *powers, cudaStream_t s);
int powers_info(const char *path, int64_t *info, int cap);
int powers_load(const char *path, int16_t *powers, int64_t cap_slots, cudaStream_t s);
int dense_minplus_noalloc(const void *X, const void *Y, void *Z, int64_t M, int64_t N,
                          int64_t K, int64_t ldx, int64_t ldy, int64_t ldz, int dtype,
                          cudaStream_t s);
int batched_run(const mp_problem *probs, int count, int mode, cudaStream_t s);
int batch_prepare(const mp_problem *probs, int count, mp_batch **out);
int batch_run(mp_batch *b, int mode, cudaStream_t s);
int batch_destroy(mp_batch *b);
int autotune(int32_t *table_out);
int tuning_set(const int32_t *table);
int tuning_get(int32_t *table);

// ------------------------------------------------------------------ errors
static thread_local char g_err[1024] = "";

int set_error(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return code;
}
const char *last_error() { return g_err; }

// ------------------------------------------------------- per-device state
static std::mutex g_mu;

constexpr int kChainStreams = 8;  // streams on which several chains run side by side

struct DeviceState {
    DeviceInfo info;
    int *status = nullptr;            // device-side error latch
    cudaStream_t sync_stream = nullptr;  // for the synchronous entry points
    cudaStream_t chain_streams[kChainStreams] = {};
};
static std::map<int, DeviceState> g_dev;

static int device_state(DeviceState **out) {
    int dev = -1;
    MP_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_dev.find(dev);
    if (it == g_dev.end()) {
        DeviceState st;
        st.info.device = dev;
        MP_CUDA_TRY(cudaDeviceGetAttribute(&st.info.sms, cudaDevAttrMultiProcessorCount, dev));
        int optin = 0;
        MP_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        st.info.smem_optin = (size_t)optin;
        int per_sm = 0;
        MP_CUDA_TRY(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
        st.info.smem_sm = (size_t)per_sm;
        MP_CUDA_TRY(cudaMalloc(&st.status, sizeof(int)));
        MP_CUDA_TRY(cudaMemset(st.status, 0, sizeof(int)));
        MP_CUDA_TRY(cudaStreamCreateWithFlags(&st.sync_stream, cudaStreamNonBlocking));
        // The library's temporaries come from the device's default memory
        // pool.  It keeps up to 1/32 of the device's memory reserved between
        // calls instead of returning it at every synchronisation, so that a
        // repeated call (a full power chain stages gigabytes) does not map
        // its buffers again; large requests trim the pool first.
        {
            cudaMemPool_t pool = nullptr;
            size_t free_b = 0, total_b = 0;
            MP_CUDA_TRY(cudaDeviceGetDefaultMemPool(&pool, dev));
            MP_CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
            uint64_t keep = (uint64_t)total_b / 32;
            MP_CUDA_TRY(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
        }
        // Side-by-side chains go to these streams largest first; the first
        // streams get the highest priorities, so the CTAs of the longest
        // chain are placed on the SMs before the short chains fill the rest.
        int lo_prio = 0, hi_prio = 0;
        MP_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio));
        for (int i = 0; i < kChainStreams; ++i)
            MP_CUDA_TRY(cudaStreamCreateWithPriority(&st.chain_streams[i], cudaStreamNonBlocking,
                                                     std::min(lo_prio, hi_prio + i)));
        it = g_dev.emplace(dev, st).first;
    }
    *out = &it->second;
    return MP_OK;
}

int device_info(DeviceInfo *out) {
    DeviceState *st;
    MP_TRY(device_state(&st));
    *out = st->info;
    return MP_OK;
}

int device_status_ptr(int **p) {
    DeviceState *st;
    MP_TRY(device_state(&st));
    *p = st->status;
    return MP_OK;
}

// ------------------------------------------------ transfer plans (cached)
struct TransferEntry {
    int n = 0;
    int64_t N = 0;
    std::vector<uint32_t> words;
    PlanDev plan;
    DevCsr csr;                // device CSR of A(D_n), labels as values
    size_t h2d_bytes = 0, d2h_bytes = 0;
    // what the narrow plan is built from, on first use
    HostCsr pcsr;              // rows and columns in the internal row order
    std::vector<uint16_t> pz;
    std::vector<int32_t> canon;
    PlanDev plan_narrow;       // the mirror-representative columns only
    bool have_narrow = false;
    int64_t narrow_cols = 0;
    CircuitHost circuit;       // reuse circuit of the rows (empty: none)
    CircuitCover gcover;       // covers of the global circuit (levels = 0: none)
    // the narrow plan's labelled first power and its diagonal minimum, kept
    // for the shared-memory circuit chains (which only read their P_1)
    DevBuf p1_narrow, g1_narrow;
    bool have_p1_narrow = false;
    // full powers from the narrow chain: per caller column c the buffer
    // column holding P[i][c] (bit 31 set: column c's mirror, read in row
    // R i), per caller row i its mirror row R i and its internal row, and
    // the rows i <= R i
    DevBuf mirror_col, mirror_row, mirror_inv, mirror_lead;
    int64_t mirror_nlead = 0;
    bool have_mirror = false;
};

// Lanes per row of the global circuit for a chain of `ncols` buffer columns:
// chunks of 8 L columns, at least about two per SM, from 32 to 256 columns.
static int gcircuit_lanes(int64_t ncols, int sms) {
    int W = 256;
    while (W > 32 && ncols / W < 2 * (int64_t)sms) W /= 2;
    return W / 8;
}

// A plan that only shapes the chain's buffers for the global circuit (no
// gather schedule): ncols columns kept (colpos: caller column -> buffer
// column, empty for all), rows in the internal order canon, buffer rows
// padded to 256 columns so every chunk width divides them.
static int gcircuit_plan(TransferEntry *e, const std::vector<int32_t> &colpos, int64_t ncols,
                         const std::vector<int32_t> &diagcol, PlanDev *d, cudaStream_t s) {
    DeviceInfo di;
    MP_TRY(device_info(&di));
    PlanHost ph;
    ph.N = e->N;
    ph.ldb = (ncols + 255) / 256 * 256;
    ph.nnz = e->pcsr.row_ptr[(size_t)e->N];
    ph.colconst = true;
    ph.z = e->pz;
    ph.canon = e->canon;
    ph.colpos = colpos;
    MP_TRY(plan_upload(ph, d, s, true));
    GCircuitHost gh;
    MP_TRY(gcircuit_slice_host(e->gcover, e->pz, gcircuit_lanes(ncols, di.sms), &gh));
    return gcircuit_upload(gh, diagcol, e->canon, d, s);
}

// Steps of transfer chains run on the reuse circuit where a column chunk fits
// shared memory; MP_SPARSE_CIRCUIT=0 in the environment keeps the gather
// plan for every step.
static bool circuit_enabled() {
    const char *v = getenv("MP_SPARSE_CIRCUIT");
    return !(v && v[0] == '0');
}
static std::map<std::pair<int, int>, std::unique_ptr<TransferEntry>> g_transfer;
static std::mutex g_narrow_mu;

// Builds (or finds) the sparse plan of A(D_n) on the current device.  The
// arcs come from the device arc test; the host only groups rows.
static int transfer_entry(int n, cudaStream_t s, TransferEntry **out) {
    int dev = -1;
    MP_CUDA_TRY(cudaGetDevice(&dev));
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_transfer.find({dev, n});
        if (it != g_transfer.end()) {
            *out = it->second.get();
            return MP_OK;
        }
    }
    auto e = std::make_unique<TransferEntry>();
    e->n = n;
    enumerate_words(n, &e->words);
    const int64_t N = (int64_t)e->words.size();
    e->N = N;
    std::vector<WordMasks> masks;
    word_masks(n, e->words, &masks);
    DevBuf dmask;
    MP_TRY(dmask.alloc(masks.size() * sizeof(WordMasks), s));
    MP_CUDA_TRY(cudaMemcpyAsync(dmask.p, masks.data(), masks.size() * sizeof(WordMasks),
                                cudaMemcpyHostToDevice, s));
    HostCsr csr;
    csr.N = N;
    MP_TRY(e->csr.row_ptr.alloc((size_t)(N + 1) * 8, s, true));
    int64_t *d_rp = e->csr.row_ptr.as<int64_t>();
    MP_TRY(launch_transfer_csr_count(n, dmask.as<WordMasks>(), N, d_rp, s));
    std::vector<int64_t> cnt((size_t)N);
    MP_CUDA_TRY(cudaMemcpyAsync(cnt.data(), d_rp, (size_t)N * 8, cudaMemcpyDeviceToHost, s));
    MP_CUDA_TRY(cudaStreamSynchronize(s));
    csr.row_ptr.assign((size_t)N + 1, 0);
    for (int64_t q = 0; q < N; ++q) csr.row_ptr[q + 1] = csr.row_ptr[q] + cnt[q];
    const int64_t nnz = csr.row_ptr[N];
    MP_CUDA_TRY(cudaMemcpyAsync(d_rp, csr.row_ptr.data(), (size_t)(N + 1) * 8,
                                cudaMemcpyHostToDevice, s));
    MP_TRY(e->csr.col.alloc((size_t)std::max<int64_t>(nnz, 1) * 4, s, true));
    MP_TRY(launch_transfer_csr_fill(n, dmask.as<WordMasks>(), N, d_rp, e->csr.col.as<int32_t>(), s));
    csr.col.resize((size_t)nnz);
    if (nnz)
        MP_CUDA_TRY(cudaMemcpyAsync(csr.col.data(), e->csr.col.p, (size_t)nnz * 4,
                                    cudaMemcpyDeviceToHost, s));
    MP_CUDA_TRY(cudaStreamSynchronize(s));
    // labels: number of zeros of the target word
    std::vector<uint16_t> z((size_t)N);
    for (int64_t p = 0; p < N; ++p) z[p] = (uint16_t)__builtin_popcount(masks[p].zero);
    csr.val.resize((size_t)nnz);
    for (int64_t t = 0; t < nnz; ++t) csr.val[t] = (int16_t)z[csr.col[t]];
    // The chain keeps its rows in an order of its own: words sorted by the
    // positions of their 1s, then of their 0s.  Rows with equal 1-positions
    // gather largely the same rows, so row groups of the gather plan come out
    // larger and fewer rows are staged per output row (at n = 9: 16% fewer
    // units, 14% fewer staged rows).  Row i of the internal buffers is word
    // canon[i]; columns keep the words' order, and every value written to
    // the caller (powers, diagonal minima) is placed by canon.
    std::vector<int32_t> canon((size_t)N), inv((size_t)N);
    for (int64_t i = 0; i < N; ++i) canon[i] = (int32_t)i;
    std::stable_sort(canon.begin(), canon.end(), [&](int32_t a, int32_t b) {
        return masks[a].one != masks[b].one ? masks[a].one < masks[b].one
                                            : masks[a].zero < masks[b].zero;
    });
    for (int64_t i = 0; i < N; ++i) inv[canon[i]] = (int32_t)i;
    // CSR with rows in the internal order: caller columns for the initial
    // power on the device, internal columns (gathered rows) for the plan
    HostCsr pcsr;
    pcsr.N = N;
    pcsr.row_ptr.assign((size_t)N + 1, 0);
    for (int64_t i = 0; i < N; ++i)
        pcsr.row_ptr[i + 1] = pcsr.row_ptr[i] + (csr.row_ptr[canon[i] + 1] - csr.row_ptr[canon[i]]);
    pcsr.col.resize((size_t)nnz);
    pcsr.val.resize((size_t)nnz);
    std::vector<int32_t> dcol((size_t)nnz);
    for (int64_t i = 0; i < N; ++i) {
        int64_t o = pcsr.row_ptr[i];
        for (int64_t t = csr.row_ptr[canon[i]]; t < csr.row_ptr[canon[i] + 1]; ++t, ++o) {
            dcol[o] = csr.col[t];
            pcsr.col[o] = inv[csr.col[t]];
            pcsr.val[o] = csr.val[t];
        }
    }
    // internal columns ascend within a row, as the plan expects
    for (int64_t i = 0; i < N; ++i) {
        const int64_t b = pcsr.row_ptr[i], f = pcsr.row_ptr[i + 1];
        std::vector<std::pair<int32_t, int32_t>> tmp;
        tmp.reserve((size_t)(f - b));
        for (int64_t t = b; t < f; ++t) tmp.push_back({pcsr.col[t], dcol[t]});
        std::sort(tmp.begin(), tmp.end());
        for (int64_t t = b; t < f; ++t) {
            pcsr.col[t] = tmp[(size_t)(t - b)].first;
            dcol[t] = tmp[(size_t)(t - b)].second;
            pcsr.val[t] = (int16_t)z[dcol[t]];
        }
    }
    std::vector<uint16_t> pz((size_t)N);
    for (int64_t i = 0; i < N; ++i) pz[i] = z[canon[i]];
    MP_CUDA_TRY(cudaMemcpyAsync(d_rp, pcsr.row_ptr.data(), (size_t)(N + 1) * 8,
                                cudaMemcpyHostToDevice, s));
    if (nnz)
        MP_CUDA_TRY(cudaMemcpyAsync(e->csr.col.p, dcol.data(), (size_t)nnz * 4,
                                    cudaMemcpyHostToDevice, s));
    MP_TRY(e->csr.val.alloc((size_t)std::max<int64_t>(nnz, 1) * 2, s, true));
    if (nnz)
        MP_CUDA_TRY(cudaMemcpyAsync(e->csr.val.p, pcsr.val.data(), (size_t)nnz * 2,
                                    cudaMemcpyHostToDevice, s));
    DeviceInfo di;
    MP_TRY(device_info(&di));
    const int64_t nh = (N + 7) & ~(int64_t)7;
    // The shared-memory circuit where an 8-column image (2 Nh + 1 rows of 16
    // bytes) leaves room in shared memory; past that the global circuit, on
    // covers taken from the arc rule; the gather plan where circuits are
    // switched off.
    const bool smem_circuit = circuit_enabled() && 2 * nh + 1 <= 0xFFFF &&
                              (size_t)(2 * nh + 1) * 16 + 1024 < di.smem_optin;
    const bool global_circuit = circuit_enabled() && !smem_circuit;
    e->pcsr = std::move(pcsr);
    e->pz = std::move(pz);
    e->canon = std::move(canon);
    const HostCsr &pcsr_ = e->pcsr;
    const std::vector<uint16_t> &pz_ = e->pz;
    const std::vector<int32_t> &canon_ = e->canon;
    if (global_circuit) {
        MP_TRY(circuit_cover_structured(n, e->words, canon_, pcsr_, kCircLambda, &e->gcover));
        MP_TRY(gcircuit_plan(e.get(), {}, N, canon_, &e->plan, s));
    } else {
        int cap = 0, blob_cap = 0, grid = 0;
        MP_TRY(sparse_cap_rows(&cap, &blob_cap, &grid));
        PlanHost ph;
        MP_TRY(plan_build_host(pcsr_, true, pz_, &canon_, 0, cap, blob_cap, grid, &ph));
        ph.canon = canon_;
        MP_TRY(plan_upload(ph, &e->plan, s, true));
        MP_CUDA_TRY(cudaStreamSynchronize(s));
    }
    if (smem_circuit) {
        // rows are internal, and so are the gathered rows of pcsr
        CircuitHost ch;
        MP_TRY(circuit_build_host(pcsr_, &ch));
        size_t bytes = 0;
        MP_TRY(circuit_smem_bytes(ch, &bytes));
        if (bytes > 0 && e->plan.ldb % kCircW == 0) {
            e->circuit = std::move(ch);
            MP_TRY(circuit_upload(e->circuit, pz_, canon_, canon_, &e->plan, s));
        }
    }
    e->h2d_bytes = masks.size() * sizeof(WordMasks) + (size_t)(N + 1) * 8 + (size_t)nnz * 2 +
                   e->plan.h2d_bytes;
    e->d2h_bytes = (size_t)N * 8 + (size_t)nnz * 4;
    std::lock_guard<std::mutex> lk(g_mu);
    auto &slot = g_transfer[{dev, n}];
    if (!slot) slot = std::move(e);
    *out = slot.get();
    return MP_OK;
}

// Reading each column word backwards maps correct words to correct words
// and arcs to arcs with the same label (the path P_n is symmetric, and the
// zero count does not change), so A[R q][R p] = A[q][p] for that reversal R,
// every power satisfies P_k[R q][R c] = P_k[q][c], and the diagonal entry of
// row q equals that of row R q.  With left multiplication the columns of a
// power depend only on the same columns of the previous one, so a chain that
// keeps one column of every pair {c, R c} (the one with c <= R c) still sees
// every diagonal value: the narrow plan does about half the work of a full
// one and serves every call that needs only the minimum diagonals.
static int narrow_plan(TransferEntry *te, cudaStream_t s, const PlanDev **out) {
    std::lock_guard<std::mutex> lk(g_narrow_mu);
    if (!te->have_narrow) {
        const int n = te->n;
        const int64_t N = te->N;
        std::vector<int64_t> partner;
        MP_TRY(mirror_words(n, te->words, &partner));
        std::vector<int32_t> colpos((size_t)N, -1);
        int64_t ncols = 0;
        for (int64_t c = 0; c < N; ++c)
            if (c <= partner[(size_t)c]) colpos[(size_t)c] = (int32_t)ncols++;
        // per internal row, the buffer column of its diagonal entry (or none)
        std::vector<int32_t> dcol((size_t)N);
        for (int64_t i = 0; i < N; ++i) dcol[(size_t)i] = colpos[(size_t)te->canon[(size_t)i]];
        if (te->gcover.levels > 0) {
            MP_TRY(gcircuit_plan(te, colpos, ncols, dcol, &te->plan_narrow, s));
            te->narrow_cols = ncols;
            te->have_narrow = true;
            *out = &te->plan_narrow;
            return MP_OK;
        }
        int cap = 0, blob_cap = 0, grid = 0;
        MP_TRY(sparse_cap_rows(&cap, &blob_cap, &grid));
        PlanHost ph;
        MP_TRY(plan_build_host(te->pcsr, true, te->pz, &dcol, ncols, cap, blob_cap, grid, &ph));
        ph.canon = te->canon;
        ph.colpos = colpos;
        MP_TRY(plan_upload(ph, &te->plan_narrow, s, true));
        MP_CUDA_TRY(cudaStreamSynchronize(s));
        if (te->circuit.W > 0 && te->plan_narrow.ldb % kCircW == 0) {
            MP_TRY(circuit_upload(te->circuit, te->pz, dcol, te->canon, &te->plan_narrow, s));
            std::vector<int32_t> mcol((size_t)N), mrow((size_t)N), inv((size_t)N), lead;
            for (int64_t c = 0; c < N; ++c) {
                const int64_t r = partner[(size_t)c];
                mcol[(size_t)c] = colpos[(size_t)c] >= 0 ? colpos[(size_t)c]
                                                          : (int32_t)(0x80000000u | (uint32_t)colpos[(size_t)r]);
                mrow[(size_t)c] = (int32_t)r;
                if (c <= r) lead.push_back((int32_t)c);
            }
            for (int64_t q = 0; q < N; ++q) inv[(size_t)te->canon[(size_t)q]] = (int32_t)q;
            MP_TRY(te->mirror_col.alloc((size_t)N * 4, s, true));
            MP_TRY(te->mirror_row.alloc((size_t)N * 4, s, true));
            MP_TRY(te->mirror_inv.alloc((size_t)N * 4, s, true));
            MP_TRY(te->mirror_lead.alloc(lead.size() * 4, s, true));
            MP_CUDA_TRY(cudaMemcpyAsync(te->mirror_col.p, mcol.data(), (size_t)N * 4, cudaMemcpyHostToDevice, s));
            MP_CUDA_TRY(cudaMemcpyAsync(te->mirror_row.p, mrow.data(), (size_t)N * 4, cudaMemcpyHostToDevice, s));
            MP_CUDA_TRY(cudaMemcpyAsync(te->mirror_inv.p, inv.data(), (size_t)N * 4, cudaMemcpyHostToDevice, s));
            MP_CUDA_TRY(cudaMemcpyAsync(te->mirror_lead.p, lead.data(), lead.size() * 4, cudaMemcpyHostToDevice, s));
            te->mirror_nlead = (int64_t)lead.size();
            MP_CUDA_TRY(cudaStreamSynchronize(s));  // the host vectors go out of scope
            te->have_mirror = te->plan_narrow.circuit.ready;
        }
        te->narrow_cols = ncols;
        te->have_narrow = true;
    }
    *out = &te->plan_narrow;
    return MP_OK;
}

// The labelled P_1 of the narrow plan (A in the mirror columns) and g[1],
// built once per plan on its first shared-memory circuit chain: such a chain
// copies its chunks of P_1 into shared memory and never writes the buffer,
// so later chains start from the same one.
static int narrow_first_power(TransferEntry *te, const PlanDev &plan, cudaStream_t s,
                              const uint16_t **p1, const int32_t **g1) {
    std::lock_guard<std::mutex> lk(g_narrow_mu);
    if (!te->have_p1_narrow) {
        MP_TRY(te->p1_narrow.alloc((size_t)plan.N * (size_t)plan.ldb * 2, s, true));
        MP_TRY(te->g1_narrow.alloc(sizeof(int32_t), s, true));
        MP_TRY(launch_fill_i32(te->g1_narrow.as<int32_t>(), 1, (int32_t)kInf16, s));
        MP_TRY(sparse_init_from_csr(plan, te->csr.row_ptr.as<int64_t>(), te->csr.col.as<int32_t>(),
                                    te->csr.val.as<int16_t>(), te->p1_narrow.as<uint16_t>(), nullptr,
                                    te->g1_narrow.as<int32_t>(), s));
        // other streams may use it as soon as this returns
        MP_CUDA_TRY(cudaStreamSynchronize(s));
        te->have_p1_narrow = true;
    }
    *p1 = te->p1_narrow.as<uint16_t>();
    *g1 = te->g1_narrow.as<int32_t>();
    return MP_OK;
}

// The chain over a prepared sparse plan; B0 already holds P_1.
// P_k goes to powers slot k - out_k0 and gdiag[k - out_k0] (out_k0 = 1 when
// B0 holds A itself).
static int run_sparse_chain(const PlanDev &plan, uint16_t *B0, uint16_t *B1, int k_max,
                            int16_t *powers, size_t slot, int32_t *gdiag, cudaStream_t s,
                            int out_k0 = 1) {
    // with a circuit the whole chain is one launch, each CTA keeping its
    // column chunk on chip from step to step
    if (plan.circuit.ready) {
        if (powers && k_max >= 2 && (plan.N & 1)) {
            // Rows of an odd number N of entries start at any 2-byte
            // boundary, so a CTA's 16-byte piece of half of them takes five
            // stores: the chain writes its powers in rows of the buffer's
            // width (one aligned store per piece) to a staging area, and one
            // copy pass moves them to the caller's rows (n = 9: 11.6 -> 8.7
            // ms for 200 powers).  With N even every row is 4-byte aligned
            // and the copy pass costs more than it saves (n = 8: 1.6 against
            // 2.0 ms), as it does where the staging area finds no room: the
            // chain writes the caller's rows itself.
            const size_t spow = (size_t)plan.N * (size_t)plan.ldb;
            const size_t nslots = (size_t)(k_max - out_k0 + 1);
            void *stage = nullptr;
            if (cudaMallocAsync(&stage, spow * nslots * 2, s) == cudaSuccess) {
                int16_t *st = static_cast<int16_t *>(stage);
                int rc = circuit_chain(plan, B0, k_max, st, spow, gdiag, s, out_k0, plan.ldb);
                if (rc == MP_OK)
                    rc = launch_repack_powers(st + (size_t)(2 - out_k0) * spow, plan.ldb, spow,
                                              powers + (size_t)(2 - out_k0) * slot, slot, plan.N, k_max - 1, s);
                cudaFreeAsync(stage, s);
                return rc;
            }
            cudaGetLastError();  // the failed allocation's error: not this call's
        }
        return circuit_chain(plan, B0, k_max, powers, slot, gdiag, s, out_k0);
    }
    if (plan.gcircuit.ready) return gcircuit_chain(plan, B0, B1, k_max, powers, slot, gdiag, s, out_k0);
    uint16_t *buf[2] = {B0, B1};
    for (int k = 2; k <= k_max; ++k) {
        MP_TRY(sparse_step(plan, buf[(k - 2) & 1], buf[(k - 1) & 1],
                           powers ? powers + (size_t)(k - out_k0) * slot : nullptr,
                           gdiag ? gdiag + (k - out_k0) : nullptr, s));
    }
    return MP_OK;
}

// Dense chain: P_k = P_{k-1} (x) A with the diagonal fused into the product.
static int run_dense_chain(const int16_t *A, int64_t N, int k_max, int16_t *powers,
                           int32_t *gdiag, cudaStream_t s) {
    const size_t slot = (size_t)N * (size_t)N;
    DevBuf tmp;
    if (!powers) MP_TRY(tmp.alloc(2 * slot * 2, s));
    const int16_t *prev = A;
    for (int k = 2; k <= k_max; ++k) {
        int16_t *out = powers ? powers + (size_t)(k - 1) * slot
                              : tmp.as<int16_t>() + (size_t)((k - 2) & 1) * slot;
        MP_TRY(dense_minplus(prev, A, out, N, N, N, N, N, N, MP_I16,
                             gdiag ? gdiag + (k - 1) : nullptr, s));
        prev = out;
    }
    return MP_OK;
}

// ------------------------------------------------ recurrence (Algorithms 3, 4)
struct Recurrence {
    int K = 0, r0 = 0, a = 0, b = 0, n0 = 0;
    std::vector<int32_t> gdiag;  // min diag A^k, k = 1..K
};
static std::map<std::pair<int, int>, Recurrence> g_rec;

static int diff_constant(const int16_t *X, const int16_t *Y, int64_t count, int32_t *d_out,
                         cudaStream_t s, bool *is_const, int32_t *b) {
    MP_TRY(launch_diff_const(X, Y, count, d_out, s));
    int32_t h[4];
    MP_CUDA_TRY(cudaMemcpyAsync(h, d_out, sizeof h, cudaMemcpyDeviceToHost, s));
    MP_CUDA_TRY(cudaStreamSynchronize(s));
    *is_const = h[2] == 0 && h[3] == 1 && h[0] == h[1];
    *b = h[0];
    return MP_OK;
}

// Algorithm 3 over K stored powers of A(D_n), then Algorithm 4.
static int64_t words_of(int n) {
    std::vector<uint32_t> w;
    enumerate_words(n, &w);
    return (int64_t)w.size();
}

// Free device memory for a large request: buffers of earlier calls were
// released stream-ordered into the device's memory pool, which keeps them
// reserved until it is trimmed, so wait for the stream and trim first.
static int device_free_bytes(cudaStream_t s, size_t *free_b) {
    int dev = 0;
    MP_CUDA_TRY(cudaStreamSynchronize(s));
    MP_CUDA_TRY(cudaGetDevice(&dev));
    cudaMemPool_t pool = nullptr;
    MP_CUDA_TRY(cudaDeviceGetDefaultMemPool(&pool, dev));
    MP_CUDA_TRY(cudaMemPoolTrimTo(pool, 0));
    size_t total_b = 0;
    MP_CUDA_TRY(cudaMemGetInfo(free_b, &total_b));
    return MP_OK;
}

static int transfer_recurrence(int n, int K, Recurrence *out, cudaStream_t s) {
    NvtxScope nv("mp_transfer_recurrence n=%d K=%d", n, K);
    const int64_t N = words_of(n);
    const size_t mat = (size_t)N * (size_t)N;
    size_t free_b = 0;
    MP_TRY(device_free_bytes(s, &free_b));
    if ((double)mat * 2.0 * (K + 3) > 0.9 * (double)free_b)
        return set_error(MP_ENOMEM, "%d powers of N = %lld do not fit the free device memory", K,
                         (long long)N);
    TransferEntry *te;
    MP_TRY(transfer_entry(n, s, &te));
    DevBuf P, g, d;
    MP_TRY(P.alloc(mat * 2 * (size_t)K, s));
    MP_TRY(g.alloc(sizeof(int32_t) * (size_t)K, s));
    MP_TRY(d.alloc(sizeof(int32_t) * 4, s));
    MP_TRY(mp_transfer_power_sequence(n, K, P.as<int16_t>(), g.as<int32_t>(), s));
    Recurrence r;
    r.K = K;
    r.gdiag.resize((size_t)K);
    MP_CUDA_TRY(cudaMemcpyAsync(r.gdiag.data(), g.p, sizeof(int32_t) * (size_t)K,
                                cudaMemcpyDeviceToHost, s));
    auto pw = [&](int k) { return P.as<int16_t>() + (size_t)(k - 1) * mat; };
    bool found = false;
    for (int i = K; i >= 1 && !found; --i)
        for (int j = i - 1; j >= 1; --j) {
            bool c;
            int32_t b;
            MP_TRY(diff_constant(pw(i), pw(j), (int64_t)mat, d.as<int32_t>(), s, &c, &b));
            if (c) {
                r.a = i - j;
                r.b = b;
                r.r0 = j;
                found = true;
                break;
            }
        }
    if (found) {
        r.n0 = -1;
        for (int i = r.r0 + r.a; i >= r.a + 1; --i) {
            bool c;
            int32_t b;
            MP_TRY(diff_constant(pw(i), pw(i - r.a), (int64_t)mat, d.as<int32_t>(), s, &c, &b));
            if (!c || b != r.b) break;
            r.n0 = i - r.a;
        }
    }
    MP_CUDA_TRY(cudaStreamSynchronize(s));
    *out = r;
    return MP_OK;
}

// The transfer chain with slot k-1 of the powers at powers + (k-1)*slot
// (slot >= N*N elements; the caller may pad slots for alignment).
// Columns per block for chains over column blocks: the largest multiple of
// the circuit's chunk whose `slabs` buffers of N rows take at most `frac` of
// the free device memory (at most the whole buffer).
static int block_width(const PlanDev &plan, int slabs, double frac, cudaStream_t s, int64_t *wb) {
    const int64_t W = gcircuit_chunk(plan);
    size_t free_b = 0;
    MP_TRY(device_free_bytes(s, &free_b));
    const double per_col = (double)slabs * (double)plan.N * 2.0;
    int64_t w = (int64_t)(frac * (double)free_b / per_col) / W * W;
    if (w < W) return set_error(MP_ENOMEM, "%d buffers of one %lld-column chunk do not fit", slabs, (long long)W);
    *wb = std::min(w, plan.ldb);
    return MP_OK;
}

// The chain without powers, one block of columns at a time where the two
// chain buffers of the whole (mirror-column) width do not fit: column
// chunks of a power depend only on the same chunks of the previous power,
// so each block runs the whole chain from its part of P_1, and the diagonal
// minima of the blocks fold into gdiag.
static int transfer_chain_blocked(TransferEntry *te, const PlanDev &plan, int k_max, int32_t *gdiag,
                                  cudaStream_t s) {
    int64_t wb = 0;
    MP_TRY(block_width(plan, 2, 0.8, s, &wb));
    DevBuf B;
    MP_TRY(B.alloc(2 * (size_t)plan.N * (size_t)wb * 2, s));
    uint16_t *B0 = B.as<uint16_t>(), *B1 = B0 + (size_t)plan.N * (size_t)wb;
    for (int64_t cb = 0; cb < plan.ldb; cb += wb) {
        const int64_t w = std::min(wb, plan.ldb - cb);
        MP_TRY(sparse_init_block_from_csr(plan, te->csr.row_ptr.as<int64_t>(), te->csr.col.as<int32_t>(),
                                          te->csr.val.as<int16_t>(), cb, w, B0, gdiag, s));
        MP_TRY(gcircuit_block_chain(plan, B0, B1, k_max, cb, w, gdiag, s));
    }
    return MP_OK;
}

// Every power written in the caller's layout from the narrow chain: the
// chain computes the mirror-representative columns and stages each power
// chunk by chunk (its label pass writes consecutive rows, so the stores
// coalesce), and since P_k[R i][R c] = P_k[i][c] one copy pass fills caller
// rows i and R i from their two staged rows.  Half the columns of the full
// chain; returns MP_ENOMEM, having launched nothing, without room for the
// staging area.
static int transfer_chain_mirrored(TransferEntry *te, const PlanDev &np, int k_max, int16_t *powers,
                                   size_t slot, int32_t *gdiag, cudaStream_t s) {
    const uint16_t *p1;
    const int32_t *g1;
    MP_TRY(narrow_first_power(te, np, s, &p1, &g1));
    const size_t spow = (size_t)np.N * (size_t)np.ldb;
    // the staging area also takes, before the chain, the full plan's buffer
    // that writing P_1 in the caller's layout fills on the way
    const size_t elems = std::max(spow * (size_t)k_max, (size_t)te->plan.N * (size_t)te->plan.ldb);
    void *stage = nullptr;
    if (cudaMallocAsync(&stage, elems * 2, s) != cudaSuccess) {
        cudaGetLastError();
        return MP_ENOMEM;
    }
    int16_t *st = static_cast<int16_t *>(stage);
    // P_1 = A in the caller's first slot
    int rc = sparse_init_from_csr(te->plan, te->csr.row_ptr.as<int64_t>(), te->csr.col.as<int32_t>(),
                                  te->csr.val.as<int16_t>(), reinterpret_cast<uint16_t *>(st), powers, nullptr, s);
    if (rc == MP_OK && gdiag) rc = launch_gdiag_init(&gdiag, &g1, 1, k_max, s);
    // P_k to staging slot k - 1 (chunk by chunk), then to the caller's slot k - 1
    int W = 0;
    if (rc == MP_OK) rc = circuit_chain_staged(np, p1, k_max, st, spow, gdiag, s, &W);
    if (rc == MP_OK)
        rc = launch_mirror_repack(st + spow, W, np.ldb, spow, powers + slot, slot, te->mirror_col.as<int32_t>(),
                                  te->mirror_row.as<int32_t>(), te->mirror_inv.as<int32_t>(),
                                  te->mirror_lead.as<int32_t>(), te->mirror_nlead, np.N, k_max - 1, s);
    cudaFreeAsync(stage, s);
    return rc;
}

static int transfer_chain_direct(TransferEntry *te, int k_max, int16_t *powers_opt, size_t slot,
                                 int32_t *gdiag_opt, cudaStream_t s) {
    // without powers to write, the narrow chain gives the same diagonals
    const PlanDev *pp = &te->plan;
    if (powers_opt && k_max >= 2) {
        const PlanDev *np = nullptr;
        MP_TRY(narrow_plan(te, s, &np));
        if (te->have_mirror) {
            const int rc = transfer_chain_mirrored(te, *np, k_max, powers_opt, slot, gdiag_opt, s);
            if (rc != MP_ENOMEM) return rc;
        }
    }
    if (!powers_opt) MP_TRY(narrow_plan(te, s, &pp));
    const PlanDev &plan = *pp;
    if (!powers_opt && plan.circuit.ready) {
        const uint16_t *p1;
        const int32_t *g1;
        MP_TRY(narrow_first_power(te, plan, s, &p1, &g1));
        if (gdiag_opt) MP_TRY(launch_gdiag_init(&gdiag_opt, &g1, 1, k_max, s));
        return circuit_chain(plan, p1, k_max, nullptr, 0, gdiag_opt, s);
    }
    if (gdiag_opt) MP_TRY(launch_fill_i32(gdiag_opt, k_max, (int32_t)kInf16, s));
    // large chains check the free memory first (a synchronisation, so a
    // graph capture of such a chain fails and it runs directly instead)
    const double need = 2.0 * (double)plan.N * (double)plan.ldb * 2.0;
    if (!powers_opt && plan.gcircuit.ready && need > (double)(1u << 30)) {
        size_t free_b = 0;
        MP_TRY(device_free_bytes(s, &free_b));
        if (need > 0.8 * (double)free_b) return transfer_chain_blocked(te, plan, k_max, gdiag_opt, s);
    }
    DevBuf B;
    MP_TRY(B.alloc(2 * (size_t)plan.N * (size_t)plan.ldb * 2, s));
    uint16_t *B0 = B.as<uint16_t>(), *B1 = B0 + (size_t)plan.N * (size_t)plan.ldb;
    MP_TRY(sparse_init_from_csr(plan, te->csr.row_ptr.as<int64_t>(), te->csr.col.as<int32_t>(),
                                te->csr.val.as<int16_t>(), B0, powers_opt, gdiag_opt, s));
    return run_sparse_chain(plan, B0, B1, k_max, powers_opt, slot, gdiag_opt, s);
}

// A chain repeated with the same arguments is captured once into a CUDA
// graph (the second call) and replayed from then on: one launch instead of
// k_max + 2, with the steps linked by programmatic dependencies.
struct ChainKey {
    int dev, n, k_max;
    const void *powers, *gdiag;
    size_t slot;
    bool operator<(const ChainKey &o) const {
        return std::tie(dev, n, k_max, powers, gdiag, slot) <
               std::tie(o.dev, o.n, o.k_max, o.powers, o.gdiag, o.slot);
    }
};
struct ChainGraph {
    int calls = 0;
    cudaGraphExec_t exec = nullptr;
    uint64_t last = 0;
};
static std::map<ChainKey, ChainGraph> g_chain_graphs;
static uint64_t g_chain_clock = 0;
constexpr size_t kChainGraphCap = 32;

int transfer_powers_strided(int n, int k_max, int16_t *powers_opt, size_t slot,
                            int32_t *gdiag_opt, cudaStream_t s) {
    if (k_max < 1) return set_error(MP_EINVAL, "k_max = %d < 1", k_max);
    NvtxScope nv("mp_transfer_chain n=%d k_max=%d%s", n, k_max, powers_opt ? " powers" : "");
    TransferEntry *te;
    MP_TRY(transfer_entry(n, s, &te));
    if (slot < (size_t)te->N * (size_t)te->N) return set_error(MP_EINVAL, "slot stride too small");
    if (powers_opt && gdiag_opt &&
        ranges_overlap(gdiag_opt, (size_t)k_max * 4, powers_opt, slot * 2 * (size_t)k_max))
        return set_error(MP_EALIAS, "gdiag overlaps the powers");
    int dev = -1;
    MP_CUDA_TRY(cudaGetDevice(&dev));
    const ChainKey key{dev, n, k_max, powers_opt, gdiag_opt, slot};
    cudaGraphExec_t exec = nullptr;
    bool capture = false;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (g_chain_graphs.size() > 8 * kChainGraphCap && !g_chain_graphs.count(key)) {
            // forget the oldest chain seen once and never captured
            auto victim = g_chain_graphs.end();
            for (auto it = g_chain_graphs.begin(); it != g_chain_graphs.end(); ++it)
                if (!it->second.exec && (victim == g_chain_graphs.end() || it->second.last < victim->second.last))
                    victim = it;
            if (victim != g_chain_graphs.end()) g_chain_graphs.erase(victim);
        }
        ChainGraph &cg = g_chain_graphs[key];
        cg.last = ++g_chain_clock;
        exec = cg.exec;
        capture = !exec && ++cg.calls >= 2;
    }
    // never capture while the caller's stream is itself being captured
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    MP_CUDA_TRY(cudaStreamIsCapturing(s, &cs));
    if (cs != cudaStreamCaptureStatusNone) return transfer_chain_direct(te, k_max, powers_opt, slot, gdiag_opt, s);
    if (exec) {
        MP_CUDA_TRY(cudaGraphLaunch(exec, s));
        return MP_OK;
    }
    if (!capture) return transfer_chain_direct(te, k_max, powers_opt, slot, gdiag_opt, s);
    cudaStream_t cap = nullptr;
    MP_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    MP_CUDA_TRY(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    const int rc = transfer_chain_direct(te, k_max, powers_opt, slot, gdiag_opt, cap);
    const cudaError_t ec = cudaStreamEndCapture(cap, &graph);
    cudaStreamDestroy(cap);
    if (rc != MP_OK || ec != cudaSuccess) {
        // A capture can be invalidated from outside it (another host thread
        // synchronising the whole device while it runs), and nothing of a
        // failed capture has run: the chain runs directly instead and is not
        // captured again.  A genuine error repeats there and is returned.
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        {
            std::lock_guard<std::mutex> lk(g_mu);
            g_chain_graphs[key].calls = std::numeric_limits<int>::min() / 2;
        }
        return transfer_chain_direct(te, k_max, powers_opt, slot, gdiag_opt, s);
    }
    const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
        cudaGetLastError();
        return transfer_chain_direct(te, k_max, powers_opt, slot, gdiag_opt, s);
    }
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (g_chain_graphs.size() > kChainGraphCap) {
            auto victim = g_chain_graphs.end();
            for (auto it = g_chain_graphs.begin(); it != g_chain_graphs.end(); ++it)
                if (it->second.exec && (victim == g_chain_graphs.end() || it->second.last < victim->second.last))
                    victim = it;
            if (victim != g_chain_graphs.end()) {
                cudaGraphExecDestroy(victim->second.exec);
                g_chain_graphs.erase(victim);
            }
        }
        g_chain_graphs[key].exec = exec;
    }
    MP_CUDA_TRY(cudaGraphLaunch(exec, s));
    return MP_OK;
}

// Streaming form of Algorithms 3 and 4 for path orders whose K stored powers
// do not fit: the chain keeps only the last R powers in a ring and, after
// every product P_k, compares P_k with P_{k-a} for a = 1..R-1 (smallest a
// first).  The first constant difference, at k = n0 + a, gives the least
// n0 of Algorithm 4 and the period a with its constant b (Lemma 1 carries
// it to every later power).
// The streaming detection over column blocks, for path orders whose ring
// of R powers does not fit at full width: every block runs the chain to
// k_limit with its own ring, and for each k and a < R the statistics of
// P_k - P_{k-a} (minimum, maximum, INF in one only, finite in both) are
// folded over the blocks; the first k, smallest a, whose difference is
// constant over all columns gives n0 = k - a as in the unblocked form.
static int transfer_recurrence_blocked(TransferEntry *te, const PlanDev &plan, int k_limit, int R,
                                       Recurrence *out, cudaStream_t s) {
    int64_t wb = 0;
    MP_TRY(block_width(plan, R, 0.8, s, &wb));
    DevBuf ring, g, st;
    MP_TRY(ring.alloc((size_t)R * (size_t)plan.N * (size_t)wb * 2, s));
    MP_TRY(g.alloc(sizeof(int32_t) * (size_t)k_limit, s));
    MP_TRY(st.alloc(sizeof(int32_t) * 4 * (size_t)(k_limit + 1) * (size_t)R, s));
    const size_t slab = (size_t)plan.N * (size_t)wb;
    auto slot = [&](int k) { return ring.as<uint16_t>() + (size_t)((k - 1) % R) * slab; };
    auto stat = [&](int k, int a) { return st.as<int32_t>() + 4 * ((size_t)k * (size_t)R + (size_t)a); };
    MP_TRY(launch_fill_i32(g.as<int32_t>(), k_limit, (int32_t)kInf16, s));
    MP_TRY(launch_diff_init(st.as<int32_t>(), (int64_t)(k_limit + 1) * R, s));
    for (int64_t cb = 0; cb < plan.ldb; cb += wb) {
        const int64_t w = std::min(wb, plan.ldb - cb);
        MP_TRY(sparse_init_block_from_csr(plan, te->csr.row_ptr.as<int64_t>(), te->csr.col.as<int32_t>(),
                                          te->csr.val.as<int16_t>(), cb, w, slot(1), g.as<int32_t>(), s));
        for (int k = 2; k <= k_limit; ++k) {
            MP_TRY(gcircuit_block_step(plan, slot(k - 1), slot(k), cb, w, g.as<int32_t>() + (k - 1), s));
            for (int a = 1; a < R && a < k; ++a)
                MP_TRY(launch_diff_const(reinterpret_cast<const int16_t *>(slot(k)),
                                         reinterpret_cast<const int16_t *>(slot(k - a)), (int64_t)(plan.N * w),
                                         stat(k, a), s, false));
        }
    }
    std::vector<int32_t> h((size_t)4 * (size_t)(k_limit + 1) * (size_t)R);
    MP_CUDA_TRY(cudaMemcpyAsync(h.data(), st.p, h.size() * 4, cudaMemcpyDeviceToHost, s));
    std::vector<int32_t> gh((size_t)k_limit);
    MP_CUDA_TRY(cudaMemcpyAsync(gh.data(), g.p, gh.size() * 4, cudaMemcpyDeviceToHost, s));
    MP_CUDA_TRY(cudaStreamSynchronize(s));
    Recurrence r;
    for (int k = 2; k <= k_limit && r.a == 0; ++k)
        for (int a = 1; a < R && a < k; ++a) {
            const int32_t *v = &h[4 * ((size_t)k * (size_t)R + (size_t)a)];
            if (v[2] == 0 && v[3] == 1 && v[0] == v[1]) {
                r.a = a;
                r.b = v[0];
                r.n0 = k - a;
                r.r0 = k - a;
                r.K = k;
                r.gdiag.assign(gh.begin(), gh.begin() + k);
                break;
            }
        }
    *out = r;
    return MP_OK;
}

static int transfer_recurrence_ring(int n, int k_limit, int R, Recurrence *out, cudaStream_t s) {
    NvtxScope nv("mp_transfer_recurrence_stream n=%d ring=%d", n, R);
    // The ring is the chain itself, narrow: slot (k - 1) % R holds the k-th
    // buffer z + P_k on the mirror-representative columns.  Labels cancel in
    // a difference, and a difference that is constant on those columns is
    // constant on all of them (the dropped columns repeat kept ones), so
    // Algorithm 3's test runs on the slots directly and no full power is
    // ever written.
    const int64_t N = words_of(n);
    const double cols_est = 0.5625 * (double)N + 64.0;  // a little over N / 2
    size_t free_b = 0;
    MP_TRY(device_free_bytes(s, &free_b));
    const bool fits = (double)N * cols_est * 2.0 * R <= 0.9 * (double)free_b;
    TransferEntry *te;
    MP_TRY(transfer_entry(n, s, &te));
    const PlanDev *pp = nullptr;
    MP_TRY(narrow_plan(te, s, &pp));
    const PlanDev &plan = *pp;
    if (plan.gcircuit.ready) {
        // the global circuit runs the ring over column blocks where it does not fit
        MP_TRY(device_free_bytes(s, &free_b));
        if ((double)plan.N * (double)plan.ldb * 2.0 * R > 0.8 * (double)free_b)
            return transfer_recurrence_blocked(te, plan, k_limit, R, out, s);
    } else if (!fits) {
        return set_error(MP_ENOMEM, "a ring of %d powers of N = %lld does not fit the free memory", R,
                         (long long)N);
    }
    const size_t slab = (size_t)plan.N * (size_t)plan.ldb;
    DevBuf ring, g, d;
    MP_TRY(ring.alloc(slab * 2 * (size_t)R, s));
    MP_TRY(g.alloc(sizeof(int32_t) * (size_t)k_limit, s));
    MP_TRY(d.alloc(sizeof(int32_t) * 4, s));
    auto slot = [&](int k) { return ring.as<uint16_t>() + (size_t)((k - 1) % R) * slab; };
    MP_TRY(launch_fill_i32(g.as<int32_t>(), k_limit, (int32_t)kInf16, s));
    MP_TRY(sparse_init_from_csr(plan, te->csr.row_ptr.as<int64_t>(), te->csr.col.as<int32_t>(),
                                te->csr.val.as<int16_t>(), slot(1), nullptr, g.as<int32_t>(), s));
    Recurrence r;
    bool found = false;
    for (int k = 2; k <= k_limit && !found; ++k) {
        MP_TRY(sparse_step(plan, slot(k - 1), slot(k), nullptr, g.as<int32_t>() + (k - 1), s));
        for (int a = 1; a < R && a < k; ++a) {
            bool c;
            int32_t b;
            MP_TRY(diff_constant(reinterpret_cast<const int16_t *>(slot(k)),
                                 reinterpret_cast<const int16_t *>(slot(k - a)), (int64_t)slab,
                                 d.as<int32_t>(), s, &c, &b));
            if (c) {
                r.a = a;
                r.b = b;
                r.n0 = k - a;
                r.r0 = k - a;
                r.K = k;
                found = true;
                break;
            }
        }
    }
    if (found) {
        r.gdiag.resize((size_t)r.K);
        MP_CUDA_TRY(cudaMemcpyAsync(r.gdiag.data(), g.p, sizeof(int32_t) * (size_t)r.K,
                                    cudaMemcpyDeviceToHost, s));
    }
    MP_CUDA_TRY(cudaStreamSynchronize(s));
    *out = r;
    return MP_OK;
}

// Repeated squaring (Theorem 2 with the power algebra of Lemma 1):
// S_0 = A, S_j = S_{j-1} (x) S_{j-1} = A^(2^j), and A^m is the product of the
// S_j over the set bits j of m.  The highest factor enters only through the
// min-trace min_{i,l} R_il + S_li, which is min diag (R (x) S) without forming
// the product.  Dense products on the DPX kernel; four N x N buffers.
// Synchronous on s; m >= 3 and m * n below the INF code (checked by callers).
static int gamma2_by_squaring(TransferEntry *te, int64_t m, cudaStream_t s, int32_t *result) {
    NvtxScope nv("mp_gamma2_squaring n=%d m=%lld", te->n, (long long)m);
    const int64_t N = te->N;
    const size_t mat = (size_t)N * (size_t)N;
    DevBuf buf, g;
    MP_TRY(buf.alloc(4 * mat * 2, s));
    MP_TRY(g.alloc(sizeof(int32_t), s));
    int16_t *S = buf.as<int16_t>(), *S2 = S + mat, *R = S + 2 * mat, *R2 = S + 3 * mat;
    std::vector<WordMasks> masks;
    word_masks(te->n, te->words, &masks);
    DevBuf dm;
    MP_TRY(dm.alloc(masks.size() * sizeof(WordMasks), s));
    MP_CUDA_TRY(cudaMemcpyAsync(dm.p, masks.data(), masks.size() * sizeof(WordMasks),
                                cudaMemcpyHostToDevice, s));
    MP_TRY(launch_build_transfer(te->n, dm.as<WordMasks>(), N, S, N, s));
    int top = 0;
    while ((m >> (top + 1)) != 0) ++top;
    if ((m & (m - 1)) == 0) {
        // m = 2^top: A^m = S_{top-1} (x) S_{top-1}
        for (int j = 0; j + 1 < top; ++j) {
            MP_TRY(dense_minplus(S, S, S2, N, N, N, N, N, N, MP_I16, nullptr, s));
            std::swap(S, S2);
        }
        MP_TRY(launch_min_trace(S, S, N, N, N, g.as<int32_t>(), s));
    } else {
        // R collects the factors of the set bits below the top one
        bool have_r = false;
        for (int j = 0; j <= top; ++j) {
            if ((m >> j) & 1) {
                if (j == top) {
                    MP_TRY(launch_min_trace(R, S, N, N, N, g.as<int32_t>(), s));
                    break;
                }
                if (!have_r) {
                    MP_CUDA_TRY(cudaMemcpyAsync(R, S, mat * 2, cudaMemcpyDeviceToDevice, s));
                    have_r = true;
                } else {
                    MP_TRY(dense_minplus(R, S, R2, N, N, N, N, N, N, MP_I16, nullptr, s));
                    std::swap(R, R2);
                }
            }
            MP_TRY(dense_minplus(S, S, S2, N, N, N, N, N, N, MP_I16, nullptr, s));
            std::swap(S, S2);
        }
    }
    MP_CUDA_TRY(cudaMemcpyAsync(result, g.as<int32_t>(), 4, cudaMemcpyDeviceToHost, s));
    // the host masks were copied from pageable memory; the result is read here
    MP_CUDA_TRY(cudaStreamSynchronize(s));
    return MP_OK;
}

// The chain resumed from a caller's power P_k0 (caller layout): the
// labelled buffer is built from it and the steps run as from A, with P_k
// written to output slot k - k0 - 1.  Without powers to write, the narrow
// plan's mirror-representative columns are taken from P_k0.
static int transfer_chain_resume(TransferEntry *te, int k0, const int16_t *Pk0, int k_max,
                                 int16_t *powers_opt, int32_t *gdiag_opt, cudaStream_t s) {
    const PlanDev *pp = &te->plan;
    DevBuf cm;
    int64_t ncols = te->N;
    if (!powers_opt) {
        MP_TRY(narrow_plan(te, s, &pp));
        std::vector<int64_t> partner;
        MP_TRY(mirror_words(te->n, te->words, &partner));
        std::vector<int32_t> colmap;
        for (int64_t c = 0; c < te->N; ++c)
            if (c <= partner[(size_t)c]) colmap.push_back((int32_t)c);
        ncols = (int64_t)colmap.size();
        MP_TRY(cm.alloc(colmap.size() * 4, s));
        MP_CUDA_TRY(cudaMemcpyAsync(cm.p, colmap.data(), colmap.size() * 4, cudaMemcpyHostToDevice, s));
        MP_CUDA_TRY(cudaStreamSynchronize(s));  // the host map goes out of scope
    }
    const PlanDev &plan = *pp;
    const int steps = k_max - k0;
    if (gdiag_opt) MP_TRY(launch_fill_i32(gdiag_opt, steps, (int32_t)kInf16, s));
    DevBuf B;
    MP_TRY(B.alloc(2 * (size_t)plan.N * (size_t)plan.ldb * 2, s));
    uint16_t *B0 = B.as<uint16_t>(), *B1 = B0 + (size_t)plan.N * (size_t)plan.ldb;
    MP_TRY(sparse_init_from_power(plan, Pk0, cm.as<int32_t>(), ncols, B0, s));
    // B0 plays A^1 of the chain: its step k makes A^(k0 + k - 1), slot k - 2
    return run_sparse_chain(plan, B0, B1, steps + 1, powers_opt, (size_t)plan.N * (size_t)plan.N,
                            gdiag_opt, s, 2);
}

static int check_n(int n) {
    if (n < 1 || n > MP_MAX_PATH_ORDER)
        return set_error(MP_EINVAL, "path order n = %d outside [1, %d]", n, MP_MAX_PATH_ORDER);
    return MP_OK;
}

}  // namespace mp

using namespace mp;

extern "C" {

const char *mp_last_error(void) { return mp::last_error(); }

int64_t mp_transfer_size(int n) {
    MP_TRY(check_n(n));
    std::vector<uint32_t> w;
    enumerate_words(n, &w);
    return (int64_t)w.size();
}

int64_t mp_transfer_words(int n, uint32_t *words, int64_t cap) {
    MP_TRY(check_n(n));
    std::vector<uint32_t> w;
    enumerate_words(n, &w);
    if (words && cap > 0)
        memcpy(words, w.data(), sizeof(uint32_t) * (size_t)std::min<int64_t>(cap, (int64_t)w.size()));
    return (int64_t)w.size();
}

int mp_transfer_circuit_info(int n, int64_t *info, int cap) {
    MP_TRY(check_n(n));
    if (!info || cap < 0) return set_error(MP_EINVAL, "info buffer missing");
    TransferEntry *te;
    MP_TRY(transfer_entry(n, nullptr, &te));
    MP_CUDA_TRY(cudaStreamSynchronize(nullptr));
    const CircuitHost &c = te->circuit;
    const GCircuitDev &g = te->plan.gcircuit;
    const int64_t v[6] = {g.ready ? 8 * g.L : c.W, g.ready ? g.levels : c.levels,
                          g.ready ? g.reads : c.reads, g.ready ? g.cover_reads : c.cover_reads,
                          te->plan.nnz, te->N};
    const int k = std::min(cap, 6);
    for (int i = 0; i < k; ++i) info[i] = v[i];
    return k;
}

int mp_build_transfer_matrix(int n, int16_t *A, int64_t lda, uint32_t *words_opt, void *stream) {
    MP_TRY(check_n(n));
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<uint32_t> w;
    enumerate_words(n, &w);
    const int64_t N = (int64_t)w.size();
    if (!A) return set_error(MP_EINVAL, "A is NULL");
    if (lda < N) return set_error(MP_EINVAL, "lda = %lld < N = %lld", (long long)lda, (long long)N);
    if (words_opt && ranges_overlap(words_opt, (size_t)N * 4, A, span_bytes(N, N, lda, 2)))
        return set_error(MP_EALIAS, "words_opt overlaps A");
    std::vector<WordMasks> masks;
    word_masks(n, w, &masks);
    DevBuf dm;
    MP_TRY(dm.alloc(masks.size() * sizeof(WordMasks), s));
    MP_CUDA_TRY(cudaMemcpyAsync(dm.p, masks.data(), masks.size() * sizeof(WordMasks),
                                cudaMemcpyHostToDevice, s));
    if (words_opt)
        MP_CUDA_TRY(cudaMemcpyAsync(words_opt, w.data(), (size_t)N * 4, cudaMemcpyHostToDevice, s));
    MP_TRY(launch_build_transfer(n, dm.as<WordMasks>(), N, A, lda, s));
    // the host vectors must outlive the pageable copies' staging
    MP_CUDA_TRY(cudaStreamSynchronize(s));
    return MP_OK;
}

int mp_minplus_mul(const void *X, const void *Y, void *Z, int64_t M, int64_t N, int64_t K,
                   int64_t ldx, int64_t ldy, int64_t ldz, int dtype, void *stream) {
    if (dtype != MP_I16 && dtype != MP_U8) return set_error(MP_EINVAL, "dtype %d", dtype);
    if (M < 0 || N < 0 || K < 0) return set_error(MP_EINVAL, "negative size");
    if (M == 0 || N == 0) return MP_OK;
    if (!Z || (K > 0 && (!X || !Y))) return set_error(MP_EINVAL, "NULL matrix pointer");
    if (ldx < std::max<int64_t>(K, 1) || ldy < N || ldz < N)
        return set_error(MP_EINVAL, "leading dimension too small");
    const size_t e = dtype == MP_I16 ? 2 : 1;
    const size_t zb = span_bytes(M, N, ldz, e);
    if (ranges_overlap(Z, zb, X, span_bytes(M, K, ldx, e)) ||
        ranges_overlap(Z, zb, Y, span_bytes(K, N, ldy, e)))
        return set_error(MP_EALIAS, "Z overlaps X or Y");
    return dense_minplus(X, Y, Z, M, N, K, ldx, ldy, ldz, dtype, nullptr, (cudaStream_t)stream);
}

int mp_minplus_mul_noalloc(const void *X, const void *Y, void *Z, int64_t M, int64_t N,
                           int64_t K, int64_t ldx, int64_t ldy, int64_t ldz, int dtype,
                           void *stream) {
    if (dtype != MP_I16 && dtype != MP_U8) return set_error(MP_EINVAL, "dtype %d", dtype);
    if (M < 0 || N < 0 || K < 0) return set_error(MP_EINVAL, "negative size");
    if (M == 0 || N == 0) return MP_OK;
    if (!Z || (K > 0 && (!X || !Y))) return set_error(MP_EINVAL, "NULL matrix pointer");
    if (ldx < std::max<int64_t>(K, 1) || ldy < N || ldz < N)
        return set_error(MP_EINVAL, "leading dimension too small");
    const size_t e = dtype == MP_I16 ? 2 : 1;
    const size_t zb = span_bytes(M, N, ldz, e);
    if (ranges_overlap(Z, zb, X, span_bytes(M, K, ldx, e)) ||
        ranges_overlap(Z, zb, Y, span_bytes(K, N, ldy, e)))
        return set_error(MP_EALIAS, "Z overlaps X or Y");
    return dense_minplus_noalloc(X, Y, Z, M, N, K, ldx, ldy, ldz, dtype, (cudaStream_t)stream);
}

int mp_minplus_power_sequence(const int16_t *A, int64_t N, int k_max, int16_t *powers_opt,
                              int32_t *gdiag_opt, void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
    if (!A || N < 1 || k_max < 1) return set_error(MP_EINVAL, "need A, N >= 1, k_max >= 1");
    const size_t abytes = (size_t)N * (size_t)N * 2;
    if (powers_opt && ranges_overlap(powers_opt, abytes * (size_t)k_max, A, abytes))
        return set_error(MP_EALIAS, "powers overlap A");
    if (gdiag_opt && (ranges_overlap(gdiag_opt, (size_t)k_max * 4, A, abytes) ||
                      (powers_opt && ranges_overlap(gdiag_opt, (size_t)k_max * 4, powers_opt,
                                                    abytes * (size_t)k_max))))
        return set_error(MP_EALIAS, "gdiag overlaps A or the powers");
    if (gdiag_opt) MP_TRY(launch_fill_i32(gdiag_opt, k_max, (int32_t)kInf16, s));

    HostCsr csr;
    DevCsr dcsr;
    MP_TRY(dense_to_csr(A, N, &csr, &dcsr, s));
    const int64_t nnz = csr.row_ptr[N];
    const bool sparse = (double)nnz <= 0.25 * (double)N * (double)N;
    if (!sparse) {
        if (powers_opt)
            MP_CUDA_TRY(cudaMemcpyAsync(powers_opt, A, abytes, cudaMemcpyDeviceToDevice, s));
        if (gdiag_opt) MP_TRY(launch_diag_min(A, N, N, gdiag_opt, false, s));
        return run_dense_chain(A, N, k_max, powers_opt, gdiag_opt, s);
    }
    // column-constant labels allow the pre-added, min-only gather
    std::vector<int32_t> zc((size_t)N, -1);
    bool colconst = true;
    for (int64_t t = 0; t < nnz && colconst; ++t) {
        int32_t &zz = zc[csr.col[t]];
        if (zz < 0) zz = csr.val[t];
        else if (zz != csr.val[t]) colconst = false;
    }
    std::vector<uint16_t> z((size_t)N, 0);
    if (colconst)
        for (int64_t p = 0; p < N; ++p) z[p] = (uint16_t)std::max(zc[p], 0);
    int cap = 0, blob_cap = 0, grid = 0;
    MP_TRY(sparse_cap_rows(&cap, &blob_cap, &grid));
    PlanHost ph;
    MP_TRY(plan_build_host(csr, colconst, z, nullptr, 0, cap, blob_cap, grid, &ph));
    PlanDev plan;
    MP_TRY(plan_upload(ph, &plan, s, false));
    DevBuf B;
    MP_TRY(B.alloc(2 * (size_t)plan.N * (size_t)plan.ldb * 2, s));
    uint16_t *B0 = B.as<uint16_t>(), *B1 = B0 + (size_t)plan.N * (size_t)plan.ldb;
    MP_TRY(sparse_init_from_dense(plan, A, B0, powers_opt, gdiag_opt, s));
    MP_TRY(run_sparse_chain(plan, B0, B1, k_max, powers_opt, (size_t)N * (size_t)N, gdiag_opt, s));
    // the host-side plan vectors were copied from pageable memory: make sure
    // the copies are done before they go out of scope
    MP_CUDA_TRY(cudaStreamSynchronize(s));
    return MP_OK;
}

int mp_transfer_power_sequence(int n, int k_max, int16_t *powers_opt, int32_t *gdiag_opt,
                               void *stream) {
    MP_TRY(check_n(n));
    std::vector<uint32_t> w;
    enumerate_words(n, &w);
    const size_t N = w.size();
    return transfer_powers_strided(n, k_max, powers_opt, N * N, gdiag_opt, (cudaStream_t)stream);
}

// Several transfer chains at once: each runs on a library stream of its own,
// forked from and joined back into the caller's stream, so the small chains'
// per-step latency overlaps the large ones' work.
int mp_transfer_power_sequences(const int *ns, int count, int k_max, int32_t *gdiag,
                                void *stream) {
    if (count < 0 || (count > 0 && (!ns || !gdiag)) || k_max < 1)
        return set_error(MP_EINVAL, "need count >= 0, the path orders, gdiag and k_max >= 1");
    for (int i = 0; i < count; ++i) MP_TRY(check_n(ns[i]));
    cudaStream_t s = (cudaStream_t)stream;
    if (count == 1) return mp_transfer_power_sequence(ns[0], k_max, nullptr, gdiag, s);
    for (int i = 0; i < count; ++i)
        for (int j = 0; j < i; ++j)
            if (ns[i] == ns[j])
                return set_error(MP_EINVAL, "path order %d appears twice", ns[i]);
    DeviceState *st;
    MP_TRY(device_state(&st));
    // largest chains first, so they take their SMs before the small ones
    std::vector<int> order((size_t)count);
    for (int i = 0; i < count; ++i) order[(size_t)i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return ns[a] > ns[b]; });
    // Chains that all run on the shared-memory circuit go into one launch,
    // the longest chain's CTAs first (separate launches on several streams
    // reach the SMs in no fixed order, and a short chain placed first can
    // push the longest one into a second wave).
    if (count <= 8 && k_max >= 2) {
        std::vector<TransferEntry *> tes;
        std::vector<const PlanDev *> plans;
        bool all = true;
        for (int k = 0; k < count && all; ++k) {
            TransferEntry *te;
            MP_TRY(transfer_entry(ns[order[(size_t)k]], s, &te));
            const PlanDev *pp = nullptr;
            MP_TRY(narrow_plan(te, s, &pp));
            all = pp->circuit.ready;
            tes.push_back(te);
            plans.push_back(pp);
        }
        if (all) {
            NvtxScope nv("mp_transfer_power_sequences %d chains, one launch", count);
            std::vector<const uint16_t *> p1((size_t)count);
            std::vector<const int32_t *> g1((size_t)count);
            std::vector<int32_t *> gd((size_t)count);
            for (int k = 0; k < count; ++k) {
                MP_TRY(narrow_first_power(tes[(size_t)k], *plans[(size_t)k], s, &p1[(size_t)k], &g1[(size_t)k]));
                gd[(size_t)k] = gdiag + (size_t)order[(size_t)k] * (size_t)k_max;
            }
            MP_TRY(launch_gdiag_init(gd.data(), g1.data(), count, k_max, s));
            return circuit_multi_chain(plans.data(), p1.data(), count, k_max, gd.data(), s);
        }
    }
    cudaEvent_t fork = nullptr;
    MP_CUDA_TRY(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    int rc = MP_OK;
    if (cudaEventRecord(fork, s) != cudaSuccess) rc = set_error(MP_ECUDA, "event record failed");
    std::vector<cudaEvent_t> joins;
    for (int k = 0; k < count && rc == MP_OK; ++k) {
        const int i = order[(size_t)k];
        cudaStream_t cs = st->chain_streams[k % kChainStreams];
        if (cudaStreamWaitEvent(cs, fork, 0) != cudaSuccess) {
            rc = set_error(MP_ECUDA, "stream wait failed");
            break;
        }
        rc = mp_transfer_power_sequence(ns[i], k_max, nullptr, gdiag + (size_t)i * (size_t)k_max, cs);
        cudaEvent_t j = nullptr;
        if (cudaEventCreateWithFlags(&j, cudaEventDisableTiming) != cudaSuccess) {
            rc = set_error(MP_ECUDA, "event create failed");
            break;
        }
        joins.push_back(j);
        // join even after a failed launch, so the caller's stream stays ordered
        if (cudaEventRecord(j, cs) != cudaSuccess || cudaStreamWaitEvent(s, j, 0) != cudaSuccess)
            rc = rc != MP_OK ? rc : set_error(MP_ECUDA, "stream join failed");
    }
    for (cudaEvent_t j : joins) cudaEventDestroy(j);
    cudaEventDestroy(fork);
    return rc;
}

int mp_gamma2_tables(const int *ns, int count, int k_max, int64_t *out) {
    if (count < 0 || (count > 0 && (!ns || !out)) || k_max < 3)
        return set_error(MP_EINVAL, "need count >= 0, the path orders, out and k_max >= 3");
    for (int i = 0; i < count; ++i) {
        MP_TRY(check_n(ns[i]));
        if ((int64_t)k_max * ns[i] >= (int64_t)kInf16)
            return set_error(MP_ERANGE, "k_max * n = %lld reaches the int16 INF code",
                             (long long)k_max * ns[i]);
    }
    if (count == 0) return MP_OK;
    DeviceState *st;
    MP_TRY(device_state(&st));
    cudaStream_t s = st->sync_stream;
    DevBuf g;
    const size_t cells = (size_t)count * (size_t)k_max;
    MP_TRY(g.alloc(sizeof(int32_t) * cells, s));
    MP_TRY(mp_transfer_power_sequences(ns, count, k_max, g.as<int32_t>(), s));
    std::vector<int32_t> h(cells);
    MP_CUDA_TRY(cudaMemcpyAsync(h.data(), g.p, sizeof(int32_t) * cells, cudaMemcpyDeviceToHost, s));
    MP_CUDA_TRY(cudaStreamSynchronize(s));
    for (int i = 0; i < count; ++i)
        for (int m = 0; m <= k_max; ++m)
            out[(size_t)i * (size_t)(k_max + 1) + (size_t)m] =
                m < 3 ? -1 : (int64_t)h[(size_t)i * (size_t)k_max + (size_t)m - 1];
    return MP_OK;
}

int mp_gamma2_table(int n, int k_max, int64_t *out) {
    MP_TRY(check_n(n));
    if (k_max < 3 || !out) return set_error(MP_EINVAL, "need k_max >= 3 and an output array");
    if ((int64_t)k_max * n >= (int64_t)kInf16)
        return set_error(MP_ERANGE, "k_max * n = %lld reaches the int16 INF code",
                         (long long)k_max * n);
    DeviceState *st;
    MP_TRY(device_state(&st));
    cudaStream_t s = st->sync_stream;
    DevBuf g;
    MP_TRY(g.alloc(sizeof(int32_t) * (size_t)k_max, s));
    MP_TRY(mp_transfer_power_sequence(n, k_max, nullptr, g.as<int32_t>(), s));
    std::vector<int32_t> h((size_t)k_max);
    MP_CUDA_TRY(cudaMemcpyAsync(h.data(), g.p, sizeof(int32_t) * (size_t)k_max,
                                cudaMemcpyDeviceToHost, s));
    MP_CUDA_TRY(cudaStreamSynchronize(s));
    for (int m = 0; m <= k_max; ++m) out[m] = m < 3 ? -1 : (int64_t)h[(size_t)m - 1];
    return MP_OK;
}

int mp_diff_const(const int16_t *X, const int16_t *Y, int64_t count, int32_t *out, void *stream) {
    if (!X || !Y || !out || count < 0) return set_error(MP_EINVAL, "bad diff_const arguments");
    return launch_diff_const(X, Y, count, out, (cudaStream_t)stream);
}

int mp_transfer_recurrence(int n, int K, int32_t *out) {
    MP_TRY(check_n(n));
    if (K < 2 || !out) return set_error(MP_EINVAL, "need K >= 2 and an output array");
    if ((int64_t)K * n >= (int64_t)kInf16)
        return set_error(MP_ERANGE, "K * n reaches the int16 INF code");
    DeviceState *st;
    MP_TRY(device_state(&st));
    Recurrence r;
    MP_TRY(transfer_recurrence(n, K, &r, st->sync_stream));
    if (r.a > 0 && r.n0 >= 1) {
        int dev = -1;
        MP_CUDA_TRY(cudaGetDevice(&dev));
        std::lock_guard<std::mutex> lk(g_mu);
        g_rec[{dev, n}] = r;
    }
    out[0] = r.r0;
    out[1] = r.a;
    out[2] = r.b;
    out[3] = r.n0;
    return MP_OK;
}

int mp_transfer_recurrence_stream(int n, int k_limit, int ring, int32_t *out) {
    MP_TRY(check_n(n));
    if (k_limit < 2 || ring < 2 || !out)
        return set_error(MP_EINVAL, "need k_limit >= 2, ring >= 2 and an output array");
    if ((int64_t)k_limit * n >= (int64_t)kInf16)
        return set_error(MP_ERANGE, "k_limit * n reaches the int16 INF code");
    DeviceState *st;
    MP_TRY(device_state(&st));
    Recurrence r;
    MP_TRY(transfer_recurrence_ring(n, k_limit, ring, &r, st->sync_stream));
    if (r.a > 0) {
        int dev = -1;
        MP_CUDA_TRY(cudaGetDevice(&dev));
        std::lock_guard<std::mutex> lk(g_mu);
        g_rec[{dev, n}] = r;
    }
    out[0] = r.n0;
    out[1] = r.a;
    out[2] = r.b;
    out[3] = r.K;
    return MP_OK;
}

int mp_diag_min(const int16_t *P, int64_t N, int64_t ld, int32_t *out, void *stream) {
    if (!P || !out || N < 0 || ld < N) return set_error(MP_EINVAL, "bad diag_min arguments");
    return launch_diag_min(P, N, ld, out, true, (cudaStream_t)stream);
}

int mp_min_trace(const int16_t *X, const int16_t *Y, int64_t N, int64_t ldx, int64_t ldy,
                 int32_t *out, void *stream) {
    if (!X || !Y || !out || N < 0 || ldx < N || ldy < N)
        return set_error(MP_EINVAL, "bad min_trace arguments");
    return launch_min_trace(X, Y, N, ldx, ldy, out, (cudaStream_t)stream);
}

int mp_gamma2_cylinder(int n, int64_t m, int64_t *out) {
    MP_TRY(check_n(n));
    if (m < 3) return set_error(MP_EINVAL, "cycle length m = %lld < 3", (long long)m);
    if (!out) return set_error(MP_EINVAL, "out is NULL");
    DeviceState *st;
    MP_TRY(device_state(&st));
    cudaStream_t s = st->sync_stream;
    // Theorem 3: with A^{n0+a} = b + A^{n0}, gamma_2(m + a) = gamma_2(m) + b for
    // m >= n0, so every m past the stored powers reduces to one of them.
    {
        int dev = -1;
        MP_CUDA_TRY(cudaGetDevice(&dev));
        Recurrence r;
        bool have = false;
        {
            std::lock_guard<std::mutex> lk(g_mu);
            auto it = g_rec.find({dev, n});
            if (it != g_rec.end()) {
                r = it->second;
                have = true;
            }
        }
        if (!have && m > 64) {
            int32_t tmp[4];
            const int rc = n <= 11 ? mp_transfer_recurrence(n, 50, tmp)
                                   : mp_transfer_recurrence_stream(n, 64, 20, tmp);
            if (rc == MP_OK) {
                std::lock_guard<std::mutex> lk(g_mu);
                auto it = g_rec.find({dev, n});
                if (it != g_rec.end()) {
                    r = it->second;
                    have = true;
                }
            }
        }
        if (have) {
            if (m <= r.K) {
                *out = r.gdiag[(size_t)m - 1];
                return MP_OK;
            }
            const int64_t t = (m - r.n0) / r.a;  // m - t*a in [n0, n0 + a)
            *out = (int64_t)r.gdiag[(size_t)(m - t * r.a) - 1] + t * (int64_t)r.b;
            return MP_OK;
        }
    }
    if (m * (int64_t)n >= (int64_t)kInf16)
        return set_error(MP_ERANGE, "m * n = %lld reaches the int16 INF code",
                         (long long)(m * n));
    TransferEntry *te;
    MP_TRY(transfer_entry(n, s, &te));
    const int64_t N = te->N;
    // cost model: chain = m steps of N*nnz terms; squaring = ~2 log2(m) dense N^3 products
    const double chain_cost = (double)m * (double)N * (double)te->plan.nnz;
    const double lg = std::floor(std::log2((double)m)) + 1.0;
    const double square_cost = 2.5 * (2.0 * lg) * (double)N * (double)N * (double)N;
    if (chain_cost > square_cost && N * N * 2 * 4 <= (int64_t)64 << 30) {
        int32_t result = 0;
        MP_TRY(gamma2_by_squaring(te, m, s, &result));
        *out = result;
        return MP_OK;
    }
    DevBuf g;
    MP_TRY(g.alloc(sizeof(int32_t) * (size_t)m, s));
    int32_t result = 0;
    MP_TRY(mp_transfer_power_sequence(n, (int)m, nullptr, g.as<int32_t>(), s));
    MP_CUDA_TRY(cudaMemcpyAsync(&result, g.as<int32_t>() + (m - 1), 4, cudaMemcpyDeviceToHost, s));
    MP_CUDA_TRY(cudaStreamSynchronize(s));
    *out = result;
    return MP_OK;
}

int mp_gamma2_squaring(int n, int64_t m, int64_t *out) {
    MP_TRY(check_n(n));
    if (m < 3) return set_error(MP_EINVAL, "cycle length m = %lld < 3", (long long)m);
    if (!out) return set_error(MP_EINVAL, "out is NULL");
    if (m * (int64_t)n >= (int64_t)kInf16)
        return set_error(MP_ERANGE, "m * n = %lld reaches the int16 INF code",
                         (long long)(m * n));
    DeviceState *st;
    MP_TRY(device_state(&st));
    cudaStream_t s = st->sync_stream;
    TransferEntry *te;
    MP_TRY(transfer_entry(n, s, &te));
    int32_t result = 0;
    MP_TRY(gamma2_by_squaring(te, m, s, &result));
    *out = result;
    return MP_OK;
}

int mp_minplus_mul_batched(const mp_problem *probs, int count, int mode, void *stream) {
    if (count < 0 || (count > 0 && !probs)) return set_error(MP_EINVAL, "bad problem list");
    if (mode != 0 && mode != 1) return set_error(MP_EINVAL, "mode %d", mode);
    return batched_run(probs, count, mode, (cudaStream_t)stream);
}

int mp_batch_prepare(const mp_problem *probs, int count, mp_batch **out) {
    if (!out) return set_error(MP_EINVAL, "out is NULL");
    *out = nullptr;
    return batch_prepare(probs, count, out);
}

int mp_batch_run(mp_batch *batch, int mode, void *stream) {
    return batch_run(batch, mode, (cudaStream_t)stream);
}

int mp_batch_destroy(mp_batch *batch) { return batch_destroy(batch); }

int mp_autotune(int32_t *table_out) { return autotune(table_out); }

int mp_tuning_set(const int32_t *table) {
    if (!table) return set_error(MP_EINVAL, "table is NULL");
    return tuning_set(table);
}

int mp_tuning_get(int32_t *table) {
    if (!table) return set_error(MP_EINVAL, "table is NULL");
    return tuning_get(table);
}

int mp_dpx_peak(int variant, int64_t iters, double *ops_per_s) {
    if (!ops_per_s) return set_error(MP_EINVAL, "ops_per_s is NULL");
    return dpx_peak(variant, iters, ops_per_s);
}

int mp_powers_save(const char *path, int n, int k0, int64_t count, const int16_t *powers, void *stream) {
    MP_TRY(check_n(n));
    if (!path || k0 < 1 || count < 0 || (count > 0 && !powers))
        return set_error(MP_EINVAL, "need a path, k0 >= 1, count >= 0 and the powers");
    return powers_save(path, n, k0, count, powers, (cudaStream_t)stream);
}

int mp_powers_info(const char *path, int64_t *info, int cap) {
    if (!path || !info || cap < 0) return set_error(MP_EINVAL, "need a path and an info array");
    return powers_info(path, info, cap);
}

int mp_powers_load(const char *path, int16_t *powers, int64_t cap_slots, void *stream) {
    if (!path || (cap_slots > 0 && !powers) || cap_slots < 0)
        return set_error(MP_EINVAL, "need a path and a buffer");
    return powers_load(path, powers, cap_slots, (cudaStream_t)stream);
}

int mp_transfer_power_sequence_from(int n, int k0, const int16_t *P_k0, int k_max, int16_t *powers_opt,
                                    int32_t *gdiag_opt, void *stream) {
    MP_TRY(check_n(n));
    if (!P_k0 || k0 < 1 || k_max <= k0)
        return set_error(MP_EINVAL, "need the power P_k0, k0 >= 1 and k_max > k0");
    cudaStream_t s = (cudaStream_t)stream;
    TransferEntry *te;
    MP_TRY(transfer_entry(n, s, &te));
    const size_t mat = (size_t)te->N * (size_t)te->N * 2;
    const size_t steps = (size_t)(k_max - k0);
    if (powers_opt && ranges_overlap(powers_opt, mat * steps, P_k0, mat))
        return set_error(MP_EALIAS, "powers overlap P_k0");
    if (gdiag_opt && (ranges_overlap(gdiag_opt, steps * 4, P_k0, mat) ||
                      (powers_opt && ranges_overlap(gdiag_opt, steps * 4, powers_opt, mat * steps))))
        return set_error(MP_EALIAS, "gdiag overlaps P_k0 or the powers");
    NvtxScope nv("mp_transfer_chain_from n=%d k0=%d k_max=%d", n, k0, k_max);
    return transfer_chain_resume(te, k0, P_k0, k_max, powers_opt, gdiag_opt, s);
}

int mp_inject_circuit_timeout(int n, void *stream) {
    MP_TRY(check_n(n));
    cudaStream_t s = (cudaStream_t)stream;
    TransferEntry *te;
    MP_TRY(transfer_entry(n, s, &te));
    const PlanDev &plan = te->plan;
    if (!plan.circuit.ready) return set_error(MP_EINVAL, "path order %d has no circuit", n);
    // valid buffers for the step's reads (the chunk of X is staged before the
    // wait); nothing is written to them
    DevBuf B;
    const size_t elems = (size_t)plan.N * (size_t)plan.ldb;
    MP_TRY(B.alloc(2 * elems * 2, s));
    MP_CUDA_TRY(cudaMemsetAsync(B.p, 0, 2 * elems * 2, s));
    return circuit_timeout_probe(plan, B.as<uint16_t>(), B.as<uint16_t>() + elems, s);
}

int mp_device_status(void) {
    DeviceState *st;
    MP_TRY(device_state(&st));
    MP_CUDA_TRY(cudaDeviceSynchronize());
    int v = 0;
    MP_CUDA_TRY(cudaMemcpy(&v, st->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (v != 0) {
        MP_CUDA_TRY(cudaMemset(st->status, 0, sizeof(int)));
        return set_error(v, v == MP_ECHECK ? "a bounds check caught an index outside its buffer"
                                           : "a device-side bounded wait ran out");
    }
    return MP_OK;
}

}  // extern "C"
