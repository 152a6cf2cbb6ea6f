// a1 + a2: correct n-words and the 2-domination transfer matrix A(D_n).
//
// Words (Section 2.2): letters 0, 1, 2; a word is correct when it contains
// none of 020, 111, 211, 112, 212, does not start with 11 or 12 and does not
// end with 11 or 21.  They are generated depth-first, letter by letter in
// the order 0 < 1 < 2, pruning a prefix as soon as it contains a forbidden
// window, so the output is in lexicographic order without a filter pass.
//
// Arcs (Section 2.2, three bullets) are tested on the device for all N^2
// pairs at once in bit-sliced form: for each word the positions holding 0,
// 1 and 2 are three n-bit masks, and the "neighbours equal to 0" counts of
// every position come from shifted masks.
#include <map>

#include "mp_internal.cuh"

namespace mp {

static void words_dfs(int n, int pos, uint32_t code, int l2, int l1,
                      std::vector<uint32_t> *out) {
    if (pos == n) {
        out->push_back(code);
        return;
    }
    for (int c = 0; c < 3; ++c) {
        if (pos >= 2) {
            // forbidden windows 020, 111, 211, 112, 212 ending at pos
            if (l2 == 0 && l1 == 2 && c == 0) continue;
            if (l1 == 1 && c == 1 && (l2 == 1 || l2 == 2)) continue;
            if (l1 == 1 && c == 2 && (l2 == 1 || l2 == 2)) continue;
        }
        if (pos == 1 && l1 == 1 && (c == 1 || c == 2)) continue;        // 11, 12 at the start
        if (pos == n - 1 && n >= 2 && c == 1 && (l1 == 1 || l1 == 2)) continue;  // 11, 21 at the end
        words_dfs(n, pos + 1, (code << 2) | (uint32_t)c, l1, c, out);
    }
}

void enumerate_words(int n, std::vector<uint32_t> *out) {
    out->clear();
    if (n < 1 || n > MP_MAX_PATH_ORDER) return;
    words_dfs(n, 0, 0u, -1, -1, out);
}

void word_masks(int n, const std::vector<uint32_t> &words, std::vector<WordMasks> *out) {
    out->resize(words.size());
    for (size_t t = 0; t < words.size(); ++t) {
        WordMasks m{0, 0, 0, 0};
        for (int i = 0; i < n; ++i) {
            uint32_t letter = (words[t] >> (2 * (n - 1 - i))) & 3u;
            uint16_t bit = (uint16_t)(1u << i);
            if (letter == 0) m.zero |= bit;
            else if (letter == 1) m.one |= bit;
            else m.two |= bit;
        }
        (*out)[t] = m;
    }
}

// Reading a word backwards keeps it correct (the forbidden windows and the
// end rules are mirror images of each other), so reversal is an involution
// on the correct words; partner[c] is the index of word c read backwards.
int mirror_words(int n, const std::vector<uint32_t> &words, std::vector<int64_t> *partner) {
    std::map<uint32_t, int64_t> index;
    for (size_t c = 0; c < words.size(); ++c) index[words[c]] = (int64_t)c;
    partner->assign(words.size(), -1);
    for (size_t c = 0; c < words.size(); ++c) {
        uint32_t r = 0;
        for (int i = 0; i < n; ++i) r |= ((words[c] >> (2 * i)) & 3u) << (2 * (n - 1 - i));
        auto it = index.find(r);
        if (it == index.end()) return set_error(MP_EINVAL, "reversed word not correct (n = %d)", n);
        (*partner)[c] = it->second;
    }
    return MP_OK;
}

// Arc q -> p ("p can follow q") in bit-sliced form.  Bit i is letter i+1.
__device__ __forceinline__ bool arc_ok(WordMasks q, WordMasks p, uint32_t full) {
    // q_i = 2 forces p_i = 0
    if (q.two & ~p.zero) return false;
    uint32_t left = ((uint32_t)p.zero << 1) & full;  // p_{i-1} = 0
    uint32_t right = (uint32_t)p.zero >> 1;          // p_{i+1} = 0
    uint32_t prev = q.zero;                          // q_i = 0
    uint32_t any2 = (left & right) | (left & prev) | (right & prev);  // >= 2 zeros
    uint32_t odd = left ^ right ^ prev;
    uint32_t exactly1 = odd & ~(left & right & prev);
    if (p.two & ~exactly1) return false;  // p_i = 2 needs exactly one zero
    if (p.one & ~any2) return false;      // p_i = 1 needs at least two zeros
    return true;
}

__global__ void build_transfer_kernel(const WordMasks *__restrict__ masks, int64_t N,
                                      int64_t q0, uint32_t full, int16_t *__restrict__ A,
                                      int64_t lda) {
    int64_t q = q0 + blockIdx.y;
    if (q >= N) return;
    WordMasks wq = masks[q];
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N;
         p += (int64_t)gridDim.x * blockDim.x) {
        WordMasks wp = masks[p];
        int16_t v = arc_ok(wq, wp, full) ? (int16_t)__popc(wp.zero) : (int16_t)kInf16;
        A[q * lda + p] = v;
    }
}

int launch_build_transfer(int n, const WordMasks *d_masks, int64_t N, int16_t *A,
                          int64_t lda, cudaStream_t s) {
    if (N <= 0) return MP_OK;
    uint32_t full = (n >= 32) ? 0xFFFFFFFFu : ((1u << n) - 1u);
    int threads = 256;
    int64_t bx = (N + threads - 1) / threads;
    if (bx > 64) bx = 64;
    for (int64_t q0 = 0; q0 < N; q0 += 65535) {
        int64_t rows = N - q0 < 65535 ? N - q0 : 65535;
        dim3 grid((unsigned)bx, (unsigned)rows);
        build_transfer_kernel<<<grid, threads, 0, s>>>(d_masks, N, q0, full, A, lda);
    }
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}

// CSR of A(D_n) straight from the words: one warp per source row q, ballots
// over 32 targets p at a time.  Pass 1 counts the arcs of each row; pass 2
// writes the target indices in increasing order (ballot prefix counts keep
// the order), so row q lists Out(q) sorted.
__global__ void transfer_csr_count_kernel(const WordMasks *__restrict__ masks, int64_t N,
                                          uint32_t full, int64_t *__restrict__ counts) {
    const int lane = threadIdx.x & 31;
    const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (q >= N) return;
    WordMasks wq = masks[q];
    int64_t c = 0;
    for (int64_t p0 = 0; p0 < N; p0 += 32) {
        int64_t p = p0 + lane;
        bool ok = p < N && arc_ok(wq, masks[p], full);
        c += __popc(__ballot_sync(0xFFFFFFFFu, ok));
    }
    if (lane == 0) counts[q] = c;
}

__global__ void transfer_csr_fill_kernel(const WordMasks *__restrict__ masks, int64_t N,
                                         uint32_t full, const int64_t *__restrict__ row_ptr,
                                         int32_t *__restrict__ col) {
    const int lane = threadIdx.x & 31;
    const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (q >= N) return;
    WordMasks wq = masks[q];
    int64_t pos = row_ptr[q];
    for (int64_t p0 = 0; p0 < N; p0 += 32) {
        int64_t p = p0 + lane;
        bool ok = p < N && arc_ok(wq, masks[p], full);
        uint32_t bal = __ballot_sync(0xFFFFFFFFu, ok);
        if (ok) col[pos + __popc(bal & ((1u << lane) - 1u))] = (int32_t)p;
        pos += __popc(bal);
    }
}

int launch_transfer_csr_count(int n, const WordMasks *d_masks, int64_t N, int64_t *counts,
                              cudaStream_t s) {
    if (N <= 0) return MP_OK;
    uint32_t full = (1u << n) - 1u;
    int64_t blocks = (N * 32 + 255) / 256;
    transfer_csr_count_kernel<<<(unsigned)blocks, 256, 0, s>>>(d_masks, N, full, counts);
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}

int launch_transfer_csr_fill(int n, const WordMasks *d_masks, int64_t N, const int64_t *row_ptr,
                             int32_t *col, cudaStream_t s) {
    if (N <= 0) return MP_OK;
    uint32_t full = (1u << n) - 1u;
    int64_t blocks = (N * 32 + 255) / 256;
    transfer_csr_fill_kernel<<<(unsigned)blocks, 256, 0, s>>>(d_masks, N, full, row_ptr, col);
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}

}  // namespace mp
