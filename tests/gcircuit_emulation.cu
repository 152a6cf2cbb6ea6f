// CPU check of the global-memory reuse circuit (host logic only, no GPU).
// Builds A(D_n) with rows in the library's internal order (words sorted by
// the positions of their 1-letters, then of their 0-letters; columns keep
// the words' order), takes the covers from the arc rule and the warp tasks
// with the library's own host code, and runs the power chain on the CPU
// with the kernel's semantics: levels in order; every row of a warp task the
// minimum over its entries, where a pad entry reads nothing, a cover entry
// reads a row of the result computed at an earlier level, and a direct
// entry reads a row of the previous power plus the label carried in the
// entry (which must be the zero count of that row's word).  The buffers hold
// the powers unlabelled.  Every row must be computed exactly once.  Powers
// P_1..P_k go to stdout as raw int16 in the caller's order; statistics to
// stderr.
//
// usage: gcircuit_emulation n k lanes_per_row
#include <cstdarg>
#include <cstdio>
#include <string>

#include "../paper_2409_17688_gb300/csrc/gcircuit.cu"

namespace mp {
int set_error(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vfprintf(stderr, fmt, ap);
    va_end(ap);
    fputc('\n', stderr);
    return code;
}
int device_info(DeviceInfo *o) {
    o->device = 0;
    o->sms = 1;
    o->smem_optin = 0;
    return MP_OK;
}
int device_status_ptr(int **p) {
    *p = nullptr;
    return MP_OK;
}
}  // namespace mp

using namespace mp;

static bool arc(const std::vector<WordMasks> &m, int64_t q, int64_t p, uint32_t full) {
    // the arc rule in the library's bit-sliced form, restated for the host
    const WordMasks a = m[q], b = m[p];
    if (a.two & ~b.zero) return false;
    const uint32_t left = ((uint32_t)b.zero << 1) & full, right = (uint32_t)b.zero >> 1, prev = a.zero;
    const uint32_t any2 = (left & right) | (left & prev) | (right & prev);
    const uint32_t one = (left ^ right ^ prev) & ~(left & right & prev);
    return !(b.two & ~one) && !(b.one & ~any2);
}

int main(int argc, char **argv) {
    if (argc < 4) return 2;
    const int n = atoi(argv[1]), kmax = atoi(argv[2]), L = atoi(argv[3]);
    std::vector<uint32_t> words;
    enumerate_words(n, &words);
    std::vector<WordMasks> masks;
    word_masks(n, words, &masks);
    const int64_t N = (int64_t)words.size();
    const uint32_t full = (1u << n) - 1u;
    std::vector<int32_t> canon((size_t)N), inv((size_t)N);
    for (int64_t i = 0; i < N; ++i) canon[(size_t)i] = (int32_t)i;
    std::stable_sort(canon.begin(), canon.end(), [&](int32_t a, int32_t b) {
        return masks[a].one != masks[b].one ? masks[a].one < masks[b].one : masks[a].zero < masks[b].zero;
    });
    for (int64_t i = 0; i < N; ++i) inv[(size_t)canon[(size_t)i]] = (int32_t)i;
    std::vector<uint16_t> z((size_t)N), pz((size_t)N);
    for (int64_t p = 0; p < N; ++p) z[(size_t)p] = (uint16_t)__builtin_popcount(masks[p].zero);
    for (int64_t i = 0; i < N; ++i) pz[(size_t)i] = z[(size_t)canon[(size_t)i]];
    // CSR in the internal order: rows and gathered rows internal
    HostCsr pcsr;
    pcsr.N = N;
    pcsr.row_ptr.push_back(0);
    for (int64_t i = 0; i < N; ++i) {
        std::vector<int32_t> cols;
        for (int64_t p = 0; p < N; ++p)
            if (arc(masks, canon[(size_t)i], p, full)) cols.push_back(inv[(size_t)p]);
        std::sort(cols.begin(), cols.end());
        for (int32_t c : cols) {
            pcsr.col.push_back(c);
            pcsr.val.push_back((int16_t)pz[(size_t)c]);
        }
        pcsr.row_ptr.push_back((int64_t)pcsr.col.size());
    }
    CircuitCover cv;
    if (circuit_cover_structured(n, words, canon, pcsr, kCircLambda, &cv) != MP_OK) return 3;
    GCircuitHost G;
    if (gcircuit_slice_host(cv, pz, L, &G) != MP_OK) return 3;
    fprintf(stderr, "levels %d tasks %zu reads %lld cover %lld nnz %lld\n", G.levels,
            G.tasks.size() / (size_t)(32 / L), (long long)G.reads, (long long)G.cover_reads,
            (long long)pcsr.row_ptr[N]);
    const int RPT = 32 / L;
    if (G.tasks.size() % (size_t)RPT || G.level_task0.back() * (size_t)RPT != G.tasks.size()) return 11;
    const uint32_t INF = 0x7FFF;
    // P_1 = A: internal rows, the caller's columns
    std::vector<uint32_t> X((size_t)(N * N), INF), R((size_t)(N * N), INF);
    for (int64_t i = 0; i < N; ++i)
        for (int64_t e = pcsr.row_ptr[i]; e < pcsr.row_ptr[i + 1]; ++e)
            X[(size_t)(i * N + canon[(size_t)pcsr.col[e]])] = pz[(size_t)pcsr.col[e]];
    std::vector<int16_t> out((size_t)(N * N));
    auto emit = [&](const std::vector<uint32_t> &B) {
        for (int64_t i = 0; i < N; ++i)
            for (int64_t c = 0; c < N; ++c) out[(size_t)(canon[(size_t)i] * N + c)] = (int16_t)B[(size_t)(i * N + c)];
        fwrite(out.data(), 2, out.size(), stdout);
    };
    emit(X);
    for (int k = 2; k <= kmax; ++k) {
        std::vector<int> done((size_t)N, -1);
        for (int l = 0; l < G.levels; ++l)
            for (uint32_t t = G.level_task0[(size_t)l]; t < G.level_task0[(size_t)l + 1]; ++t) {
                uint32_t tmax = G.tasks[(size_t)t * RPT].tmax4;
                for (int r = 0; r < RPT; ++r) {
                    const GCircuitHost::Slot &d = G.tasks[(size_t)t * RPT + (size_t)r];
                    if (d.tmax4 != tmax || d.len4 > tmax) return 12;  // the task's bound is uniform
                    if (d.row == 0xFFFFFFFFu) {
                        if (d.len4 != 0) return 13;
                        continue;
                    }
                    const uint32_t q = d.row;
                    if (q >= (uint32_t)N || done[q] >= 0) return 4;  // a row computed once
                    std::vector<uint32_t> acc((size_t)N, INF);
                    for (uint32_t e4 = 0; e4 < d.len4; ++e4)
                        for (int j = 0; j < 4; ++j) {
                            const uint32_t e = G.ents[((size_t)d.off4 + e4) * 4 + (size_t)j];
                            if (e & kGPad) continue;
                            const uint32_t row = e & kGRow;
                            if (row >= (uint32_t)N) return 6;
                            if (e & kGCover) {
                                if (done[row] < 0 || done[row] >= l) return 5;  // read after its level
                                for (int64_t c = 0; c < N; ++c)
                                    acc[(size_t)c] = std::min(acc[(size_t)c], R[(size_t)(row * N + c)]);
                            } else {
                                const uint32_t zl = (e >> 24) & 0xFu;
                                if (zl != pz[row]) return 8;  // the entry's label is its row's
                                for (int64_t c = 0; c < N; ++c)
                                    acc[(size_t)c] = std::min(acc[(size_t)c], X[(size_t)(row * N + c)] + zl);
                            }
                        }
                    for (int64_t c = 0; c < N; ++c) R[(size_t)(q * N + c)] = acc[(size_t)c];
                    done[q] = l;
                }
                (void)tmax;
            }
        for (int64_t q = 0; q < N; ++q)
            if (done[q] < 0) return 7;  // every row computed
        std::swap(X, R);
        emit(X);
    }
    return 0;
}
