// Checkpoints of transfer-matrix powers.  The paper keeps A and its powers
// on disk between its algorithms (Section 3: Algorithm 1 writes A, the
// later algorithms read the powers back); here a file holds a run of
// consecutive powers A^k0 .. A^(k0 + count - 1) of one path order so a long
// chain can stop and resume from its last power.
//
// File layout (little-endian, 64-byte header, then the data):
//   0  char[8]  "MPPOWERS"
//   8  uint32   format version (1)
//  12  uint32   header bytes (64)
//  16  int32    path order n
//  20  int32    k0, the exponent of the first stored power
//  24  int64    N = |C_n|
//  32  int64    count of stored powers
//  40  int32    INF code (0x7FFF)
//  44  uint32   word order (1: lexicographic, letter 1 most significant,
//               0 < 1 < 2; row and column q are the q-th word)
//  48  uint64   FNV-1a hash of the packed word list (uint32 each), so a
//               file written with another word order or rule is refused
//  56  uint64   0
//  64  int16    count x N x N entries, row-major, power by power
#include <stdio.h>
#include <string.h>

#include <vector>

#include "mp_internal.cuh"

namespace mp {

namespace {

constexpr char kMagic[8] = {'M', 'P', 'P', 'O', 'W', 'E', 'R', 'S'};
constexpr uint32_t kVersion = 1, kHeaderBytes = 64, kWordOrderLex = 1;
constexpr size_t kStageBytes = (size_t)64 << 20;  // pinned staging per copy

struct Header {
    char magic[8];
    uint32_t version, header_bytes;
    int32_t n, k0;
    int64_t N, count;
    int32_t inf;
    uint32_t word_order;
    uint64_t words_hash, reserved;
};
static_assert(sizeof(Header) == kHeaderBytes, "checkpoint header layout");

uint64_t words_hash(const std::vector<uint32_t> &w) {
    uint64_t h = 1469598103934665603ull;  // FNV-1a, 64 bits, over little-endian bytes
    for (uint32_t x : w)
        for (int b = 0; b < 4; ++b) {
            h ^= (x >> (8 * b)) & 0xFFu;
            h *= 1099511628211ull;
        }
    return h;
}

int read_header(FILE *f, const char *path, Header *h) {
    if (fread(h, sizeof *h, 1, f) != 1) return set_error(MP_EIO, "%s: no checkpoint header", path);
    if (memcmp(h->magic, kMagic, 8) != 0 || h->header_bytes != kHeaderBytes)
        return set_error(MP_EIO, "%s is not a powers checkpoint", path);
    if (h->version != kVersion) return set_error(MP_EIO, "%s: format version %u", path, h->version);
    if (h->n < 1 || h->n > MP_MAX_PATH_ORDER || h->count < 0 || h->k0 < 1 || h->inf != (int32_t)kInf16 ||
        h->word_order != kWordOrderLex)
        return set_error(MP_EIO, "%s: header fields out of range", path);
    std::vector<uint32_t> w;
    enumerate_words(h->n, &w);
    if (h->N != (int64_t)w.size() || h->words_hash != words_hash(w))
        return set_error(MP_EIO, "%s: its words are not this library's words of path order %d", path, h->n);
    if (fseek(f, 0, SEEK_END) != 0) return set_error(MP_EIO, "%s: cannot seek", path);
    const long long size = ftell(f);
    const long long want = (long long)kHeaderBytes + (long long)h->count * h->N * h->N * 2;
    if (size != want) return set_error(MP_EIO, "%s: %lld bytes, the header implies %lld", path, size, want);
    if (fseek(f, (long)kHeaderBytes, SEEK_SET) != 0) return set_error(MP_EIO, "%s: cannot seek", path);
    return MP_OK;
}

struct File {
    FILE *f = nullptr;
    ~File() {
        if (f) fclose(f);
    }
};
struct Pinned {
    void *p = nullptr;
    ~Pinned() {
        if (p) cudaFreeHost(p);
    }
};

}  // namespace

int powers_save(const char *path, int n, int k0, int64_t count, const int16_t *powers, cudaStream_t s) {
    std::vector<uint32_t> w;
    enumerate_words(n, &w);
    const int64_t N = (int64_t)w.size();
    Header h;
    memset(&h, 0, sizeof h);
    memcpy(h.magic, kMagic, 8);
    h.version = kVersion;
    h.header_bytes = kHeaderBytes;
    h.n = n;
    h.k0 = k0;
    h.N = N;
    h.count = count;
    h.inf = (int32_t)kInf16;
    h.word_order = kWordOrderLex;
    h.words_hash = words_hash(w);
    File f;
    f.f = fopen(path, "wb");
    if (!f.f) return set_error(MP_EIO, "cannot open %s for writing", path);
    if (fwrite(&h, sizeof h, 1, f.f) != 1) return set_error(MP_EIO, "%s: write failed", path);
    const size_t total = (size_t)count * (size_t)N * (size_t)N * 2;
    Pinned st;
    if (total) MP_CUDA_TRY(cudaMallocHost(&st.p, std::min(total, kStageBytes)));
    const uint8_t *src = reinterpret_cast<const uint8_t *>(powers);
    for (size_t o = 0; o < total; o += kStageBytes) {
        const size_t b = std::min(kStageBytes, total - o);
        MP_CUDA_TRY(cudaMemcpyAsync(st.p, src + o, b, cudaMemcpyDeviceToHost, s));
        MP_CUDA_TRY(cudaStreamSynchronize(s));
        if (fwrite(st.p, 1, b, f.f) != b) return set_error(MP_EIO, "%s: write failed", path);
    }
    if (fflush(f.f) != 0) return set_error(MP_EIO, "%s: write failed", path);
    return MP_OK;
}

int powers_info(const char *path, int64_t *info, int cap) {
    File f;
    f.f = fopen(path, "rb");
    if (!f.f) return set_error(MP_EIO, "cannot open %s", path);
    Header h;
    MP_TRY(read_header(f.f, path, &h));
    const int64_t v[4] = {h.n, h.N, h.k0, h.count};
    const int k = std::min(cap, 4);
    for (int i = 0; i < k; ++i) info[i] = v[i];
    return k;
}

int powers_load(const char *path, int16_t *powers, int64_t cap_slots, cudaStream_t s) {
    File f;
    f.f = fopen(path, "rb");
    if (!f.f) return set_error(MP_EIO, "cannot open %s", path);
    Header h;
    MP_TRY(read_header(f.f, path, &h));
    if (h.count > cap_slots)
        return set_error(MP_EINVAL, "%s holds %lld powers, the buffer %lld", path, (long long)h.count,
                         (long long)cap_slots);
    const size_t total = (size_t)h.count * (size_t)h.N * (size_t)h.N * 2;
    Pinned st;
    if (total) MP_CUDA_TRY(cudaMallocHost(&st.p, std::min(total, kStageBytes)));
    uint8_t *dst = reinterpret_cast<uint8_t *>(powers);
    for (size_t o = 0; o < total; o += kStageBytes) {
        const size_t b = std::min(kStageBytes, total - o);
        // the previous copy out of the staging buffer must be done before it is refilled
        MP_CUDA_TRY(cudaStreamSynchronize(s));
        if (fread(st.p, 1, b, f.f) != b) return set_error(MP_EIO, "%s: short read", path);
        MP_CUDA_TRY(cudaMemcpyAsync(dst + o, st.p, b, cudaMemcpyHostToDevice, s));
    }
    MP_CUDA_TRY(cudaStreamSynchronize(s));
    return MP_OK;
}

}  // namespace mp
