// CPU check of the reuse circuit of the sparse transfer step (host logic
// only, no GPU).  Builds A(D_n) and its circuit with the library's own host
// code, then runs the power chain on the CPU with the circuit's semantics:
// levels in order; in each warp slice of 32 lane tasks, every lane the
// minimum over its block of 8 entries (rows of the labelled previous power,
// rows of the result computed at an earlier level, or the INF row), the
// lanes of one row (an aligned group of 1 << lg lanes) combined, the first
// lane of the group writing the row.  Every row must be computed exactly
// once and only read after it is done.  The powers P_1..P_k go to stdout as
// raw int16 so the test can compare them with the oracle; the circuit's
// statistics go to stderr.
//
// With a fourth argument "image" the chain runs the way the chain kernel
// keeps it in shared memory instead: one image of 2Nh + 1 rows (X, the
// result from row Nh, the INF row 2Nh), entry j read at (j + sh) mod 2Nh,
// result row q written at (Nh + q + sh) mod 2Nh, the labels added in place
// after each step, and sh swapping between 0 and Nh; the rows between the
// regions must never be read.
//
// usage: circuit_emulation n k [image]
#include <cstdarg>
#include <cstdio>
#include <string>

#include "../paper_2409_17688_gb300/csrc/circuit.cu"

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
    if (argc < 3) return 2;
    const int n = atoi(argv[1]), kmax = atoi(argv[2]);
    const bool image = argc > 3 && std::string(argv[3]) == "image";
    std::vector<uint32_t> words;
    enumerate_words(n, &words);
    std::vector<WordMasks> masks;
    word_masks(n, words, &masks);
    const int64_t N = (int64_t)words.size();
    const uint32_t full = (1u << n) - 1u;
    HostCsr csr;
    csr.N = N;
    csr.row_ptr.push_back(0);
    std::vector<uint16_t> z((size_t)N);
    for (int64_t p = 0; p < N; ++p) z[p] = (uint16_t)__builtin_popcount(masks[p].zero);
    for (int64_t q = 0; q < N; ++q) {
        for (int64_t p = 0; p < N; ++p)
            if (arc(masks, q, p, full)) {
                csr.col.push_back((int32_t)p);
                csr.val.push_back((int16_t)z[p]);
            }
        csr.row_ptr.push_back((int64_t)csr.col.size());
    }
    CircuitHost C;
    if (circuit_build_host(csr, &C) != MP_OK) return 3;
    const int64_t nsl = C.level_slice0.back();
    fprintf(stderr, "levels %d slices %lld reads %lld cover %lld nnz %lld\n", C.levels, (long long)nsl,
            (long long)C.reads, (long long)C.cover_reads, (long long)csr.row_ptr[N]);
    if ((int64_t)C.info.size() != nsl * 32 || (int64_t)C.ents.size() != nsl * 32 * 8) return 11;
    const uint32_t INF = 0x7FFF;
    const uint32_t N2 = (uint32_t)(2 * C.Nh);
    std::vector<int16_t> Pk((size_t)(N * N), (int16_t)INF);
    for (int64_t q = 0; q < N; ++q)
        for (int64_t e = csr.row_ptr[q]; e < csr.row_ptr[q + 1]; ++e) Pk[q * N + csr.col[e]] = csr.val[e];
    fwrite(Pk.data(), 2, Pk.size(), stdout);
    // the lane groups of every slice: a row's lanes are an aligned group of
    // 1 << lg lanes with the same info; idle lanes hold row 0xFFFF
    for (int64_t s = 0; s < nsl; ++s)
        for (int i = 0; i < 32;) {
            const uint32_t info = C.info[(size_t)(s * 32 + i)];
            const uint32_t q = info & 0xFFFFu, g = 1u << ((info >> 16) & 7u);
            if (q == 0xFFFFu) {
                ++i;
                continue;
            }
            if (i % g || i + g > 32) return 12;
            for (uint32_t t = 0; t < g; ++t)
                if (C.info[(size_t)(s * 32 + i + t)] != info) return 13;
            // the widest row of a slice comes first (its lane 0 sets the shuffle count)
            if (g > 1u << ((C.info[(size_t)(s * 32)] >> 16) & 7u)) return 14;
            i += (int)g;
        }
    // per step: img(j) is the value of image row j at column c (labelled X
    // rows, result rows, the INF row), done[q] the level that computed q
    std::vector<uint32_t> X((size_t)(N * N)), R((size_t)(N * N));
    std::vector<uint32_t> imgbuf;
    const int64_t Nh = C.Nh;
    if (image) {
        imgbuf.assign((size_t)((N2 + 1) * N), 0xDEADu);  // gap rows: never read
        for (int64_t q = 0; q < N; ++q)
            for (int64_t c = 0; c < N; ++c) imgbuf[q * N + c] = (uint32_t)(uint16_t)Pk[q * N + c] + z[q];
        for (int64_t c = 0; c < N; ++c) imgbuf[N2 * N + c] = 0xFFFFu;
    }
    int64_t sh = 0;
    auto at = [&](int64_t j) { j += sh; return j >= N2 ? j - N2 : j; };
    for (int k = 2; k <= kmax; ++k) {
        if (!image)
            for (int64_t q = 0; q < N; ++q)  // the labelled buffer z_q + P_k[q]
                for (int64_t c = 0; c < N; ++c) X[q * N + c] = (uint32_t)(uint16_t)Pk[q * N + c] + z[q];
        std::vector<int> done((size_t)N, -1);
        for (int l = 0; l < C.levels; ++l)
            for (int64_t s = C.level_slice0[l]; s < C.level_slice0[l + 1]; ++s)
                for (int i = 0; i < 32;) {
                    const uint32_t info = C.info[(size_t)(s * 32 + i)];
                    const uint32_t q = info & 0xFFFFu, g = 1u << ((info >> 16) & 7u);
                    if (q == 0xFFFFu) {
                        for (int t = 0; t < 8; ++t)  // an idle lane loads nothing
                            if (C.ents[(size_t)(s * 32 + i) * 8 + t] != N2) return 15;
                        ++i;
                        continue;
                    }
                    if (q >= (uint32_t)N || done[q] >= 0) return 4;  // a row computed once
                    for (int64_t c = 0; c < N; ++c) {
                        uint32_t acc = INF;
                        for (uint32_t lane = 0; lane < g; ++lane)
                            for (int t = 0; t < 8; ++t) {
                                const uint32_t idx = C.ents[(size_t)(s * 32 + i + lane) * 8 + t];
                                if (idx == N2) continue;  // padding: no load
                                const bool xrow = idx < (uint32_t)N;
                                const bool rrow = idx >= (uint32_t)Nh && idx < (uint32_t)(Nh + N);
                                if (!xrow && !rrow) return 6;  // a row between the regions
                                if (rrow) {
                                    const int64_t qq = idx - Nh;
                                    if (done[qq] < 0 || done[qq] >= l) return 5;  // read after its level
                                }
                                uint32_t v;
                                if (image) {
                                    v = imgbuf[at(idx) * N + c];
                                    if (v == 0xDEADu) return 10;  // never written
                                } else {
                                    v = xrow ? X[idx * N + c] : R[(idx - Nh) * N + c];
                                }
                                acc = std::min(acc, v);
                            }
                        if (image) imgbuf[at(Nh + q) * N + c] = acc;
                        else R[q * N + c] = acc;
                        Pk[q * N + c] = (int16_t)acc;
                    }
                    done[q] = l;
                    i += (int)g;
                }
        for (int64_t q = 0; q < N; ++q)
            if (done[q] < 0) return 7;  // every row computed
        if (image) {
            for (int64_t q = 0; q < N; ++q)  // the labels, in place
                for (int64_t c = 0; c < N; ++c) imgbuf[at(Nh + q) * N + c] += z[q];
            sh = Nh - sh;
        }
        fwrite(Pk.data(), 2, Pk.size(), stdout);
    }
    return 0;
}
