// CPU check of the sparse transfer-step plan (host logic only, no GPU).
// Builds the plan of A(D_n) with the library's own host code and carries out
// the kernel's semantics on the CPU: for every unit of every CTA, each warp's
// entry stream is reduced segment by segment, the segment minima are folded
// into the rows of their cluster masks, finished tasks fold into the row
// accumulators, and the last stage of an item writes the rows.  The
// powers P_1..P_k are written to stdout as raw int16 (row-major) so the test
// can compare them with the oracle.
//
// usage: plan_emulation n k cluster_max cap_rows
#include <cstdarg>
#include <cstdio>

#include "../paper_2409_17688_gb300/csrc/spmm_plan.cu"

namespace mp {
int set_error(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vfprintf(stderr, fmt, ap);
    va_end(ap);
    fputc('\n', stderr);
    return code;
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
    if (argc < 5) return 2;
    const int n = atoi(argv[1]), kmax = atoi(argv[2]), cl = atoi(argv[3]), cap = atoi(argv[4]);
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
    PlanHost P;
    if (plan_build_host(csr, true, z, nullptr, 0, cap, 6144, 7, &P, cl) != MP_OK) return 3;
    fprintf(stderr, "groups %d stages %zu units %zu\n", P.ngroups, P.stage_u0.size() - 1,
            P.units.size());
    const int INF = 0x7FFF;
    const int64_t ldb = P.ldb;
    // B holds z_row + P_k (the kernel's pre-added layout), padding columns INF + z
    std::vector<uint32_t> B((size_t)(N * ldb)), out((size_t)(N * ldb));
    std::vector<int16_t> Pk((size_t)(N * N), (int16_t)INF);
    for (int64_t q = 0; q < N; ++q)
        for (int64_t e = csr.row_ptr[q]; e < csr.row_ptr[q + 1]; ++e) Pk[q * N + csr.col[e]] = csr.val[e];
    auto load_B = [&]() {
        for (int64_t q = 0; q < N; ++q)
            for (int64_t c = 0; c < ldb; ++c)
                B[q * ldb + c] = (uint32_t)(c < N ? (uint16_t)Pk[q * N + c] : INF) + z[q];
    };
    fwrite(Pk.data(), 2, Pk.size(), stdout);
    std::vector<uint32_t> acc((size_t)kGroupMax * kChunk, INF);
    for (int k = 2; k <= kmax; ++k) {
        load_B();
        std::fill(out.begin(), out.end(), 0xFFFFFFFFu);
        for (const UnitDesc &u : P.units) {
            const int chunk = (int)(u.meta & 0xFFFF);
            const bool last = (u.meta >> 31) != 0;
            const uint32_t *blob = P.blob.data() + (size_t)u.bo8 * 8;
            const int row0 = (int)blob[0], nrows = (int)blob[1], ntasks = (int)blob[3], nsegs = (int)blob[4];
            const uint32_t *tasks = blob + kBlobHeader;
            const uint16_t *zs = reinterpret_cast<const uint16_t *>(tasks + ((ntasks + 7) & ~7));
            const uint32_t *ents = reinterpret_cast<const uint32_t *>(zs) + ((nrows + 15) / 16) * 8 +
                                   ((nrows + 7) & ~7);
            (void)nsegs;
            for (int w = 0; w < kWarps; ++w) {
                const int e0 = (int)blob[kStreamStart + w], e1 = (int)blob[kStreamStart + w + 1];
                if ((e1 - e0) % 8 != 0 || (e0 % 4) != 0) return 5;  // whole blocks, 16-byte aligned
                for (int c = 0; c < kChunk; ++c) {
                    int t = (int)blob[8 + w];
                    uint32_t m[4] = {0xFFFFu, 0xFFFFu, 0xFFFFu, 0xFFFFu}, s = 0xFFFFu;
                    for (int e = e0; e < e1; e += 4) {  // one 4-entry block per pass
                        const uint32_t word = ents[e + 3];
                        for (int i = 0; i < 4; ++i) {
                            if ((ents[e + i] & ~kEntOffset) != (word & ~kEntOffset)) return 6;
                            const int urow = (int)((ents[e + i] & kEntOffset) / kRowBytes);
                            s = std::min(s, urow == P.cap_rows - 1
                                                ? 0xFFFFu
                                                : B[(int64_t)P.urows[u.u0 + urow] * ldb + chunk * kChunk + c]);
                        }
                        if (!(word & kEntSegEnd)) continue;
                        if ((e - e0) % 8 != 4) return 8;  // only the second block of a pair ends a segment
                        for (int j = 0; j < 4; ++j)
                            if ((word >> kEntMaskShift) & (1u << j)) m[j] = std::min(m[j], s);
                        s = 0xFFFFu;
                        if (!(word & kEntTaskEnd)) continue;
                        const uint32_t t0 = tasks[t++];
                        for (int j = 0; j < (int)(t0 >> 24); ++j) {
                            const int r = (int)((t0 >> (6 * j)) & 0x3F);
                            acc[(size_t)r * kChunk + c] = std::min(acc[(size_t)r * kChunk + c], m[j]);
                            m[j] = 0xFFFFu;
                        }
                    }
                    if (t != (int)blob[8 + w + 1]) return 7;  // every task of the warp ended
                }
            }
            if (last)
                for (int r = 0; r < nrows; ++r)
                    for (int c = 0; c < kChunk; ++c) {
                        out[(int64_t)(row0 + r) * ldb + chunk * kChunk + c] = acc[(size_t)r * kChunk + c];
                        acc[(size_t)r * kChunk + c] = INF;
                    }
        }
        for (int64_t q = 0; q < N; ++q)
            for (int64_t c = 0; c < N; ++c) {
                const uint32_t v = out[q * ldb + c];
                if (v > (uint32_t)INF) return 4;  // every output written, values in range
                Pk[q * N + c] = (int16_t)v;
            }
        fwrite(Pk.data(), 2, Pk.size(), stdout);
    }
    return 0;
}
