// Index files: hc_save writes an index's sorted lists (the output of
// Algorithm 1) to a file, hc_load reads them back over the same database, so
// that a database need not be indexed again.  The paper rebuilds its index
// from the database; this sits beside the method, off the query path.
//
// File layout, little-endian, every section a multiple of 8 bytes:
//   header   "HCURVIDX", u32 version (1), u32 byte-order mark 0x01020304,
//            u64 n, u32 d, curves, dims_per_curve, bits, dtype, partitions,
//            lists, row_bytes, flags (bit 0: low key words stored, bit 1: dim
//            map stored), u32 0, u64 total entries             (80 bytes)
//   u64 list_off[lists + 1]
//   u32 dim_map[curves * dims_per_curve] when flag bit 1, zero-padded
//   u64 keys_hi[total]
//   u64 keys_lo[total] when flag bit 0
//   u32 ids[total], zero-padded
//   u64 checksum of every 64-bit word before it (FileHash)
//
// hc_load trusts nothing in the file: the header must describe a valid index
// whose layout matches the one hc_build makes for those parameters, the size
// must match, every list must hold each row of its partition exactly once,
// high key words must not decrease along a list, the checksum must agree,
// and the keys of sampled entries, recomputed from the given database rows,
// must equal the stored ones.
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "hc_index.h"
#include "hc_trace.h"

using namespace hc;

namespace {

constexpr char kMagic[8] = {'H', 'C', 'U', 'R', 'V', 'I', 'D', 'X'};
constexpr uint32_t kVersion = 1;
constexpr uint32_t kByteOrder = 0x01020304u;
constexpr size_t kHeaderBytes = 80;
constexpr uint32_t kFlagLo = 1u, kFlagDimMap = 2u;
constexpr size_t kChunkWords = (size_t)4 << 20;   // 32 MB of host staging
constexpr uint32_t kSamplesPerList = 4096;

size_t pad8(size_t b) { return (b + 7) & ~(size_t)7; }

// Order-dependent 64-bit mix of the file's words (a damage check, not a
// cryptographic digest): h = (h xor w) * odd constant, then a right-shift fold.
struct FileHash {
    uint64_t h = 0x6a09e667f3bcc908ull;
    void words(const uint64_t* w, size_t n) {
        uint64_t x = h;
        for (size_t i = 0; i < n; ++i) {
            x = (x ^ w[i]) * 0x9e3779b97f4a7c15ull;
            x ^= x >> 29;
        }
        h = x;
    }
};

struct Header {
    uint64_t n = 0, total = 0;
    uint32_t version = 0, bom = 0, d = 0, curves = 0, m = 0, bits = 0, dtype = 0, partitions = 0,
             lists = 0, row_bytes = 0, flags = 0;
};

void put32(unsigned char* b, size_t& o, uint32_t v) { std::memcpy(b + o, &v, 4); o += 4; }
void put64(unsigned char* b, size_t& o, uint64_t v) { std::memcpy(b + o, &v, 8); o += 8; }
uint32_t get32(const unsigned char* b, size_t& o) { uint32_t v; std::memcpy(&v, b + o, 4); o += 4; return v; }
uint64_t get64(const unsigned char* b, size_t& o) { uint64_t v; std::memcpy(&v, b + o, 8); o += 8; return v; }

void encode_header(const Header& H, unsigned char (&b)[kHeaderBytes]) {
    std::memset(b, 0, kHeaderBytes);
    std::memcpy(b, kMagic, 8);
    size_t o = 8;
    put32(b, o, H.version);
    put32(b, o, H.bom);
    put64(b, o, H.n);
    put32(b, o, H.d);
    put32(b, o, H.curves);
    put32(b, o, H.m);
    put32(b, o, H.bits);
    put32(b, o, H.dtype);
    put32(b, o, H.partitions);
    put32(b, o, H.lists);
    put32(b, o, H.row_bytes);
    put32(b, o, H.flags);
    put32(b, o, 0u);
    put64(b, o, H.total);
}

bool decode_header(const unsigned char (&b)[kHeaderBytes], Header& H) {
    if (std::memcmp(b, kMagic, 8) != 0) return false;
    size_t o = 8;
    H.version = get32(b, o);
    H.bom = get32(b, o);
    H.n = get64(b, o);
    H.d = get32(b, o);
    H.curves = get32(b, o);
    H.m = get32(b, o);
    H.bits = get32(b, o);
    H.dtype = get32(b, o);
    H.partitions = get32(b, o);
    H.lists = get32(b, o);
    H.row_bytes = get32(b, o);
    H.flags = get32(b, o);
    const uint32_t zero = get32(b, o);
    H.total = get64(b, o);
    for (size_t i = o; i < kHeaderBytes; ++i)
        if (b[i]) return false;
    return H.version == kVersion && H.bom == kByteOrder && zero == 0 &&
           (H.flags & ~(kFlagLo | kFlagDimMap)) == 0;
}

// Bytes of the whole file for a header (0 when the sizes overflow).
uint64_t file_bytes(const Header& H) {
    if (H.lists > 256 || H.curves > 32 || H.m > 16 || H.total >= (1ull << 32)) return 0;
    uint64_t b = kHeaderBytes + 8ull * (H.lists + 1);
    if (H.flags & kFlagDimMap) b += pad8(4ull * H.curves * H.m);
    b += 8 * H.total;
    if (H.flags & kFlagLo) b += 8 * H.total;
    b += pad8(4 * H.total) + 8;
    return b;
}

struct FileCloser {
    FILE* f;
    ~FileCloser() {
        if (f) fclose(f);
    }
};

// ------------------------------------------------------------------ write

struct Writer {
    FILE* f;
    FileHash hash;
    bool ok = true;
    void put(const void* p, size_t bytes) {   // bytes % 8 == 0, p 8-byte aligned
        if (!ok) return;
        hash.words(static_cast<const uint64_t*>(p), bytes / 8);
        ok = fwrite(p, 1, bytes, f) == bytes;
    }
};

// Device array -> file through the host buffer, in chunks (the last one
// zero-padded to a whole word).
int save_array(Writer& w, const void* dev, size_t bytes, std::vector<uint64_t>& buf,
               cudaStream_t s) {
    const size_t chunk = buf.size() * 8;
    for (size_t o = 0; o < bytes; o += chunk) {
        const size_t b = bytes - o < chunk ? bytes - o : chunk;
        buf[(b - 1) / 8] = 0;
        if (cudaMemcpyAsync(buf.data(), static_cast<const char*>(dev) + o, b,
                            cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return HC_ERR_CUDA;
        w.put(buf.data(), pad8(b));
        if (!w.ok) return HC_ERR_IO;
    }
    return HC_OK;
}

// ------------------------------------------------------------------- read

struct Reader {
    FILE* f;
    FileHash hash;
    // HC_ERR_FORMAT at the end of the file, HC_ERR_IO on a read error
    int get(void* p, size_t bytes) {   // bytes % 8 == 0, p 8-byte aligned
        if (fread(p, 1, bytes, f) != bytes) return ferror(f) ? HC_ERR_IO : HC_ERR_FORMAT;
        hash.words(static_cast<const uint64_t*>(p), bytes / 8);
        return HC_OK;
    }
};

// Checks that stream through a section as it is read.
struct ListCursor {
    const std::vector<uint64_t>& off;   // list offsets (host)
    uint32_t list = 0;
    // advance to the list holding global entry i
    void seek(uint64_t i) {
        while (list + 1 < off.size() - 1 && i >= off[list + 1]) ++list;
    }
};

__global__ void verify_sample_kernel(IndexView ix, uint32_t per_list, uint32_t* bad) {
    const uint32_t L = blockIdx.y;
    const uint64_t off = ix.list_off[L], len = ix.list_off[L + 1] - off;
    const uint32_t c = L % ix.P.curves;
    const uint32_t want = len < per_list ? (uint32_t)len : per_list;
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < want;
         j += gridDim.x * blockDim.x) {
        // spread over the list, first and last entries included
        const uint64_t i = off + (want > 1 ? ((len - 1) * j) / (want - 1) : 0);
        const uint32_t id = ix.ids[i];
        uint64_t h, l;
        curve_key(static_cast<const uint8_t*>(ix.db) + (size_t)id * ix.row_bytes, ix.P, c, h, l);
        if (h != ix.keys_hi[i] || (ix.keys_lo && l != ix.keys_lo[i])) atomicOr(bad, 1u);
    }
}

// The sections after the header and the list offsets, checked while read.
int load_arrays(Reader& r, hc_index* x, const Header& H, cudaStream_t s) {
    std::vector<uint64_t> buf(kChunkWords);
    const uint64_t total = H.total;
    const std::vector<uint64_t>& off = x->list_off;
    // high words: ascending within each list
    {
        ListCursor cur{off};
        uint64_t prev = 0;
        for (uint64_t i0 = 0; i0 < total; i0 += kChunkWords) {
            const size_t nw = (size_t)(total - i0 < kChunkWords ? total - i0 : kChunkWords);
            if (int rc = r.get(buf.data(), 8 * nw)) return rc;
            for (size_t j = 0; j < nw; ++j) {
                const uint64_t i = i0 + j;
                cur.seek(i);
                if (i != off[cur.list] && buf[j] < prev) return HC_ERR_FORMAT;
                prev = buf[j];
            }
            if (cudaMemcpyAsync(x->keys_hi + i0, buf.data(), 8 * nw, cudaMemcpyHostToDevice, s) !=
                    cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess)
                return HC_ERR_CUDA;
        }
    }
    if (x->keys_lo) {
        for (uint64_t i0 = 0; i0 < total; i0 += kChunkWords) {
            const size_t nw = (size_t)(total - i0 < kChunkWords ? total - i0 : kChunkWords);
            if (int rc = r.get(buf.data(), 8 * nw)) return rc;
            if (cudaMemcpyAsync(x->keys_lo + i0, buf.data(), 8 * nw, cudaMemcpyHostToDevice, s) !=
                    cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess)
                return HC_ERR_CUDA;
        }
    }
    // ids: every list holds each row of its partition exactly once
    {
        const uint32_t parts = x->params.partitions;
        std::vector<uint64_t> seen;
        ListCursor cur{off};
        uint32_t list_seen = ~0u;
        uint64_t ps = 0, pe = 0;
        const uint64_t ids_per_chunk = 2 * kChunkWords;
        for (uint64_t i0 = 0; i0 < total; i0 += ids_per_chunk) {
            const uint64_t ni = total - i0 < ids_per_chunk ? total - i0 : ids_per_chunk;
            if (int rc = r.get(buf.data(), pad8(4 * ni))) return rc;
            const uint32_t* ids = reinterpret_cast<const uint32_t*>(buf.data());
            for (uint64_t j = 0; j < ni; ++j) {
                const uint64_t i = i0 + j;
                cur.seek(i);
                if (cur.list != list_seen) {
                    list_seen = cur.list;
                    const uint32_t part = cur.list / x->params.curves;
                    ps = partition_start(part, x->params.n, parts);
                    pe = partition_start(part + 1, x->params.n, parts);
                    seen.assign((pe - ps + 63) / 64, 0);
                }
                const uint64_t id = ids[j];
                if (id < ps || id >= pe) return HC_ERR_FORMAT;
                uint64_t& word = seen[(id - ps) / 64];
                const uint64_t bit = 1ull << ((id - ps) % 64);
                if (word & bit) return HC_ERR_FORMAT;
                word |= bit;
            }
            if ((ni & 1) && ids[ni] != 0) return HC_ERR_FORMAT;   // the padding
            if (cudaMemcpyAsync(x->ids + i0, buf.data(), 4 * ni, cudaMemcpyHostToDevice, s) !=
                    cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess)
                return HC_ERR_CUDA;
        }
    }
    const uint64_t expect = r.hash.h;
    uint64_t stored = 0;
    if (fread(&stored, 1, 8, r.f) != 8) return ferror(r.f) ? HC_ERR_IO : HC_ERR_FORMAT;
    if (stored != expect) return HC_ERR_FORMAT;
    return HC_OK;
}

// Recomputes sampled keys from the rows (the file must index this database).
int verify_against_rows(hc_index* x, cudaStream_t s) {
    uint32_t* bad = nullptr;
    if (cudaMallocAsync((void**)&bad, sizeof(uint32_t), s) != cudaSuccess) {
        cudaGetLastError();
        return HC_ERR_OOM;
    }
    int rc = status_of(cudaMemsetAsync(bad, 0, sizeof(uint32_t), s));
    if (!rc) {
        verify_sample_kernel<<<dim3(16, x->lists), 256, 0, s>>>(view_of(x), kSamplesPerList, bad);
        count_launches(1);
        rc = status_of(cudaGetLastError());
    }
    uint32_t h = 1;
    if (!rc) rc = status_of(cudaMemcpyAsync(&h, bad, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    cudaFreeAsync(bad, s);
    if (!rc) rc = status_of(cudaStreamSynchronize(s));
    if (!rc && h) rc = HC_ERR_FORMAT;
    return rc;
}

}  // namespace

extern "C" {

HC_API int hc_save(const hc_index* idx, const char* path, void* cuda_stream) {
    TraceRange tr("hc_save");
    if (!idx || !path) return HC_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    if (cudaStreamSynchronize(s) != cudaSuccess) return HC_ERR_CUDA;
    const hc_build_params& P = idx->params;
    Header H;
    H.version = kVersion;
    H.bom = kByteOrder;
    H.n = P.n;
    H.d = P.d;
    H.curves = P.curves;
    H.m = P.dims_per_curve;
    H.bits = P.bits;
    H.dtype = (uint32_t)P.dtype;
    H.partitions = P.partitions;
    H.lists = idx->lists;
    H.row_bytes = idx->row_bytes;
    H.flags = (idx->keys_lo ? kFlagLo : 0u) | (idx->dim_map.empty() ? 0u : kFlagDimMap);
    H.total = idx->list_off[idx->lists];

    const std::string tmp = std::string(path) + ".tmp";
    FILE* f = fopen(tmp.c_str(), "wb");
    if (!f) return HC_ERR_IO;
    int rc = HC_OK;
    {
        FileCloser fc{f};
        Writer w{f};
        alignas(8) unsigned char hb[kHeaderBytes];
        encode_header(H, hb);
        w.put(hb, kHeaderBytes);
        w.put(idx->list_off.data(), 8 * (idx->lists + 1));
        if (!idx->dim_map.empty()) {
            std::vector<uint64_t> dm(pad8(4 * idx->dim_map.size()) / 8, 0);
            std::memcpy(dm.data(), idx->dim_map.data(), 4 * idx->dim_map.size());
            w.put(dm.data(), 8 * dm.size());
        }
        if (!w.ok) rc = HC_ERR_IO;
        std::vector<uint64_t> buf(kChunkWords);
        if (!rc) rc = save_array(w, idx->keys_hi, 8 * H.total, buf, s);
        if (!rc && idx->keys_lo) rc = save_array(w, idx->keys_lo, 8 * H.total, buf, s);
        if (!rc) rc = save_array(w, idx->ids, 4 * H.total, buf, s);
        if (!rc) {
            const uint64_t h = w.hash.h;
            if (fwrite(&h, 1, 8, f) != 8) rc = HC_ERR_IO;
        }
        if (!rc && fflush(f) != 0) rc = HC_ERR_IO;
        fc.f = nullptr;
        if (fclose(f) != 0 && !rc) rc = HC_ERR_IO;
    }
    if (!rc && std::rename(tmp.c_str(), path) != 0) rc = HC_ERR_IO;
    if (rc) std::remove(tmp.c_str());
    return rc;
}

HC_API int hc_load(const char* path, const void* db_dev, void* cuda_stream, hc_index** out) {
    TraceRange tr("hc_load");
    if (!path || !out) return HC_ERR_ARG;
    *out = nullptr;
    FILE* f = fopen(path, "rb");
    if (!f) return HC_ERR_IO;
    FileCloser fc{f};
    Reader r{f};

    // the header and the list offsets, checked on the host before any device work
    alignas(8) unsigned char hb[kHeaderBytes];
    Header H;
    if (int rc = r.get(hb, kHeaderBytes)) return rc;
    if (!decode_header(hb, H)) return HC_ERR_FORMAT;
    const uint64_t want = file_bytes(H);
    if (want == 0 || fseek(f, 0, SEEK_END) != 0) return HC_ERR_FORMAT;
    const long have = ftell(f);
    if (have < 0 || (uint64_t)have != want) return HC_ERR_FORMAT;
    if (fseek(f, (long)kHeaderBytes, SEEK_SET) != 0) return HC_ERR_IO;
    std::vector<uint64_t> list_off(H.lists + 1);
    if (int rc = r.get(list_off.data(), 8 * list_off.size())) return rc;
    std::vector<uint32_t> dim_map;
    if (H.flags & kFlagDimMap) {
        std::vector<uint64_t> dm(pad8(4ull * H.curves * H.m) / 8);
        if (int rc = r.get(dm.data(), 8 * dm.size())) return rc;
        dim_map.resize((size_t)H.curves * H.m);
        std::memcpy(dim_map.data(), dm.data(), 4 * dim_map.size());
    }
    hc_build_params P{};
    P.n = H.n;
    P.d = H.d;
    P.curves = H.curves;
    P.dims_per_curve = H.m;
    P.bits = H.bits;
    P.dtype = (hc_dtype)H.dtype;
    P.dim_map = dim_map.empty() ? nullptr : dim_map.data();
    P.partitions = H.partitions;
    if (H.partitions == 0 || H.dtype > 1u) return HC_ERR_FORMAT;
    hc_index* x;
    if (index_new(db_dev, &P, out, &x) != HC_OK) return HC_ERR_FORMAT;
    index_layout(x);
    const bool lo = (H.flags & kFlagLo) != 0;
    if (x->lists != H.lists || x->row_bytes != H.row_bytes || x->list_off != list_off ||
        x->list_off[x->lists] != H.total || lo != index_keeps_lo(x->params)) {
        index_destroy(x);
        return HC_ERR_FORMAT;
    }
    if (!is_device_ptr(db_dev) || !aligned16(db_dev)) {
        index_destroy(x);
        return HC_ERR_ARG;
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int rc = index_alloc(x, s);
    if (!rc) rc = load_arrays(r, x, H, s);
    if (!rc && x->fence) rc = status_of(launch_fence(x->keys_hi, H.total, x->fence, s));
    if (!rc) rc = verify_against_rows(x, s);
    if (rc) {
        cudaStreamSynchronize(s);
        index_destroy(x);
        return rc;
    }
    *out = x;
    return HC_OK;
}

}  // extern "C"
