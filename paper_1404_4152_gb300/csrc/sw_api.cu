// Host side of the C ABI declared in include/sw.h: database loading (the
// length-sorted index of Section III), search orchestration (query profile,
// wavefront kernels, int32 rescoring, top-k: stages (i)-(iv) of the workflow
// in Section III, Fig. 2) and error reporting.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "sw.h"
#include "sw_internal.h"
#include "sw_db.h"

using namespace swgb;

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------

namespace swgb {

static thread_local std::string g_last_error;

sw_status fail(sw_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

sw_status cuda_fail(cudaError_t e, const char* what) {
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(SW_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    }
    return fail(SW_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

void clear_error() { g_last_error.clear(); }

// Device allocation against the handle's budget.
cudaError_t db_malloc(sw_db* db, void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    if (db->budget && db->dev_bytes + bytes > db->budget) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) db->dev_bytes += bytes;
    return e;
}

void db_free(sw_db* db, void* p, size_t bytes) {
    if (!p) return;
    cudaFree(p);
    if (bytes == 0) bytes = 16;
    db->dev_bytes -= std::min(db->dev_bytes, (uint64_t)bytes);
}

}  // namespace swgb

extern "C" const char* sw_last_error(void) { return g_last_error.c_str(); }
extern "C" const char* sw_version(void) { return "swgb300 0.1"; }

// ---------------------------------------------------------------------------
// database
// ---------------------------------------------------------------------------

namespace {

struct DevicePin {
    int prev = -1;
    bool ok = false;
    explicit DevicePin(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DevicePin() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

template <class T>
sw_status alloc_copy(sw_db* db, T** dst, const T* src, size_t count, cudaStream_t st,
                     const char* what) {
    void* p = nullptr;
    cudaError_t e = db_malloc(db, &p, count * sizeof(T));
    if (e != cudaSuccess) return cuda_fail(e, what);
    *dst = (T*)p;
    if (count) {
        e = cudaMemcpyAsync(p, src, count * sizeof(T), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, what);
    }
    return SW_OK;
}

void release(sw_db* db) {
    if (!db) return;
    DevicePin pin(db->device);
    for (auto& a : db->allocs) db_free(db, a.first, a.second);
    db->allocs.clear();
    if (db->stream) cudaStreamDestroy(db->stream);
    if (db->a_stream) cudaStreamDestroy(db->a_stream);
    if (db->blk_stream) cudaStreamDestroy(db->blk_stream);
    if (db->blk_fork) cudaEventDestroy(db->blk_fork);
    if (db->blk_join) cudaEventDestroy(db->blk_join);
    if (db->a_ev0) cudaEventDestroy(db->a_ev0);
    if (db->a_ev1) cudaEventDestroy(db->a_ev1);
    if (db->ev_t0) cudaEventDestroy(db->ev_t0);
    if (db->ev_t1) cudaEventDestroy(db->ev_t1);
    if (db->h_pinned) cudaFreeHost(db->h_pinned);
    if (db->graph.exec) cudaGraphExecDestroy(db->graph.exec);
    for (DevBuf* b : {&db->b_pairs, &db->b_qoff, &db->b_qlen, &db->b_flags, &db->b_topk,
                      &db->b_queries, &db->b_scores, &db->b_top, &db->a_rows, &db->a_hits,
                      &db->a_dir, &db->a_ops})
        db_free(db, b->p, b->cap);
    for (auto& t : db->pending) { cudaEventDestroy(t.a); cudaEventDestroy(t.b); }
    for (auto ev : db->event_pool) cudaEventDestroy(ev);
    delete db;
}

}  // namespace

namespace swgb {

// Tracked allocation that lives as long as the handle.
sw_status db_alloc(sw_db* db, void** p, size_t bytes, const char* what) {
    cudaError_t e = db_malloc(db, p, bytes);
    if (e != cudaSuccess) return cuda_fail(e, what);
    db->allocs.emplace_back(*p, bytes);
    return SW_OK;
}

}  // namespace swgb

extern "C" sw_status sw_db_load(const uint8_t* residues, const uint64_t* offsets,
                                uint64_t n_seqs, uint32_t alphabet, const sw_db_opts* opts,
                                sw_db** out) {
    clear_error();
    if (!out) return fail(SW_ERR_INVALID_ARG, "sw_db_load: out is NULL");
    *out = nullptr;
    if (!offsets) return fail(SW_ERR_INVALID_ARG, "sw_db_load: offsets is NULL");
    if (n_seqs == 0) return fail(SW_ERR_INVALID_ARG, "sw_db_load: n_seqs must be >= 1");
    if (n_seqs >= 0xffffffffull)
        return fail(SW_ERR_INVALID_ARG, "sw_db_load: at most 2^32-2 sequences are supported");
    if (alphabet == 0 || alphabet > SW_MAX_ALPHABET)
        return fail(SW_ERR_INVALID_ARG, "sw_db_load: alphabet must be 1..32, got %u", alphabet);
    const uint64_t total = offsets[n_seqs] - offsets[0];
    if (offsets[n_seqs] < offsets[0])
        return fail(SW_ERR_INVALID_ARG, "sw_db_load: offsets are not ascending");
    if (total && !residues) return fail(SW_ERR_INVALID_ARG, "sw_db_load: residues is NULL");

    // lengths, validated
    std::vector<uint32_t> len(n_seqs);
    uint32_t max_len = 0;
    for (uint64_t s = 0; s < n_seqs; ++s) {
        if (offsets[s + 1] < offsets[s])
            return fail(SW_ERR_INVALID_ARG, "sw_db_load: offsets not ascending at %llu",
                        (unsigned long long)s);
        const uint64_t n = offsets[s + 1] - offsets[s];
        if (n > (1u << 30))
            return fail(SW_ERR_INVALID_ARG, "sw_db_load: sequence %llu is too long",
                        (unsigned long long)s);
        len[s] = (uint32_t)n;
        max_len = std::max(max_len, (uint32_t)n);
    }

    sw_db* db = new (std::nothrow) sw_db();
    if (!db) return fail(SW_ERR_OOM, "sw_db_load: host allocation failed");
    db->device = opts ? opts->device : 0;
    db->alphabet = alphabet;
    db->n_seqs = n_seqs;
    db->total_residues = total;
    db->max_len = max_len;
    db->seq_len = len;
    db->long_threshold = (opts && opts->long_threshold) ? opts->long_threshold : 3000u;
    db->budget = opts ? opts->device_budget : 0;
    db->flags = opts ? opts->flags : 0;

    DevicePin pin(db->device);
    if (!pin.ok) {
        release(db);
        return fail(SW_ERR_CUDA, "sw_db_load: cannot select device %d", db->device);
    }
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&db->stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreate(&db->ev_t0)) != cudaSuccess ||
        (e = cudaEventCreate(&db->ev_t1)) != cudaSuccess) {
        sw_status st = cuda_fail(e, "sw_db_load: stream/event creation");
        release(db);
        return st;
    }
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, db->device);
    db->nsm = prop.multiProcessorCount;

    // Length-sorted order (descending length, ascending index among equals):
    // the offline index of Section III sorts by length for load balance; the
    // longest come first so the persistent kernels start with the biggest work.
    std::vector<uint64_t> count((size_t)max_len + 2, 0);
    for (uint64_t s = 0; s < n_seqs; ++s) ++count[max_len - len[s]];
    uint64_t acc = 0;
    for (auto& c : count) { const uint64_t v = c; c = acc; acc += v; }
    const uint64_t n_tiles = (n_seqs + kTileSeqs - 1) / kTileSeqs;
    std::vector<uint32_t> sorted(n_tiles * kTileSeqs, 0xffffffffu);
    for (uint64_t s = 0; s < n_seqs; ++s) sorted[count[max_len - len[s]]++] = (uint32_t)s;
    db->pos_of.assign(n_seqs, 0);
    for (uint64_t p = 0; p < sorted.size(); ++p)
        if (sorted[p] != 0xffffffffu) db->pos_of[sorted[p]] = (uint32_t)p;

    std::vector<uint64_t> tile_off(n_tiles);
    std::vector<uint32_t> tile_len(n_tiles);
    uint64_t off = 0;
    for (uint64_t t = 0; t < n_tiles; ++t) {
        const uint32_t first = sorted[t * kTileSeqs];
        uint32_t L = (len[first] + 3u) & ~3u;
        if (L < 4) L = 4;
        tile_len[t] = L;
        tile_off[t] = off;
        off += (uint64_t)L * kTileSeqs;
    }
    uint64_t n_long = 0;
    for (uint64_t s = 0; s < n_seqs; ++s) n_long += len[s] > db->long_threshold;
    db->n_long = n_long;
    {
        // residues per bin: the long bin is tiles [0, n_long_tiles)
        const uint64_t long_positions = ((n_long + kTileSeqs - 1) / kTileSeqs) * kTileSeqs;
        for (uint64_t p = 0; p < std::min<uint64_t>(long_positions, sorted.size()); ++p)
            if (sorted[p] != 0xffffffffu) db->residues_long += len[sorted[p]];
        db->residues_short = total - db->residues_long;
    }
    db->n_tiles = n_tiles;
    db->n_long_tiles = (n_long + kTileSeqs - 1) / kTileSeqs;
    db->tile_bytes = off;
    db->max_len_long = db->n_long_tiles ? tile_len[0] : 0;
    db->max_len_short = db->n_long_tiles < n_tiles ? tile_len[db->n_long_tiles] : 0;
    db->tile_len_host = tile_len;
    set_block_route(db, opts ? opts->block_threshold : 0);

    // device copies
    sw_status st = SW_OK;
    uint8_t* d_raw = nullptr;
    uint64_t* d_offsets = nullptr;
    std::vector<uint64_t> off0(n_seqs + 1);
    for (uint64_t s = 0; s <= n_seqs; ++s) off0[s] = offsets[s] - offsets[0];
    if ((st = alloc_copy(db, &d_raw, residues, total, db->stream, "sw_db_load: residues")) ||
        (st = alloc_copy(db, &d_offsets, off0.data(), n_seqs + 1, db->stream,
                         "sw_db_load: offsets"))) {
        db_free(db, d_raw, total);
        db_free(db, d_offsets, (n_seqs + 1) * 8);
        release(db);
        return st;
    }
    auto cleanup_raw = [&]() {
        db_free(db, d_raw, total);
        db_free(db, d_offsets, (n_seqs + 1) * 8);
    };
    // validate residue codes on the device
    uint32_t* d_max = nullptr;
    if ((st = db_alloc(db, (void**)&d_max, 64, "sw_db_load: counters"))) {
        cleanup_raw();
        release(db);
        return st;
    }
    db->d_misc = d_max;
    cudaMemsetAsync(d_max, 0, 64, db->stream);
    if ((e = launch_max_code(d_raw, total, d_max, db->stream)) != cudaSuccess) {
        st = cuda_fail(e, "sw_db_load: code check");
        cleanup_raw();
        release(db);
        return st;
    }
    uint32_t hmax = 0;
    cudaMemcpyAsync(&hmax, d_max, 4, cudaMemcpyDeviceToHost, db->stream);
    if ((e = cudaStreamSynchronize(db->stream)) != cudaSuccess) {
        st = cuda_fail(e, "sw_db_load: upload");
        cleanup_raw();
        release(db);
        return st;
    }
    if (total && hmax >= alphabet) {
        cleanup_raw();
        release(db);
        return fail(SW_ERR_INVALID_ARG, "sw_db_load: residue code %u is not below alphabet %u",
                    hmax, alphabet);
    }

    if ((st = db_alloc(db, (void**)&db->d_tile_data, db->tile_bytes, "sw_db_load: tiles")) ||
        (st = db_alloc(db, (void**)&db->d_tile_off, n_tiles * 8, "sw_db_load: tile offsets")) ||
        (st = db_alloc(db, (void**)&db->d_tile_len, n_tiles * 4, "sw_db_load: tile lengths")) ||
        (st = db_alloc(db, (void**)&db->d_sorted, n_tiles * kTileSeqs * 4,
                       "sw_db_load: sorted ids")) ||
        (st = db_alloc(db, (void**)&db->d_scores, n_seqs * 4, "sw_db_load: score buffer"))) {
        cleanup_raw();
        release(db);
        return st;
    }
    cudaMemcpyAsync(db->d_tile_off, tile_off.data(), n_tiles * 8, cudaMemcpyHostToDevice,
                    db->stream);
    cudaMemcpyAsync(db->d_tile_len, tile_len.data(), n_tiles * 4, cudaMemcpyHostToDevice,
                    db->stream);
    cudaMemcpyAsync(db->d_sorted, sorted.data(), n_tiles * kTileSeqs * 4, cudaMemcpyHostToDevice,
                    db->stream);
    e = launch_build_tiles(d_raw, d_offsets, db->d_sorted, n_tiles * kTileSeqs, db->d_tile_off,
                           db->d_tile_len, n_tiles, db->d_tile_data, db->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(db->stream);
    cleanup_raw();
    if (e != cudaSuccess) {
        st = cuda_fail(e, "sw_db_load: tile build");
        release(db);
        return st;
    }
    if ((st = sw_db_prepare_search(db))) {
        release(db);
        return st;
    }
    *out = db;
    return SW_OK;
}

extern "C" void sw_db_free(sw_db* db) { release(db); }

extern "C" sw_status sw_db_get_info(const sw_db* db, sw_db_info* info) {
    clear_error();
    if (!db || !info) return fail(SW_ERR_INVALID_ARG, "sw_db_get_info: NULL argument");
    info->n_seqs = db->n_seqs;
    info->total_residues = db->total_residues;
    info->device_bytes = db->dev_bytes;
    info->alphabet = db->alphabet;
    info->max_length = db->max_len;
    info->n_long = db->n_long;
    info->device = db->device;
    info->n_block = std::min<uint64_t>(db->n_block_tiles * kTileSeqs, db->n_seqs);
    info->block_threshold = db->block_threshold;
    return SW_OK;
}

// ---------------------------------------------------------------------------
// saving and reopening a loaded database (the offline index of Section III)
// ---------------------------------------------------------------------------

namespace {

// File layout (little-endian, as written by this library): the header below,
// then n_seqs uint32 sequence lengths (original order), n_tiles * 8 uint32
// sorted ids (sorted position -> original index, UINT32_MAX for empty slots),
// n_tiles uint32 tile lengths, and tile_bytes of tile data. Tile offsets are
// the running sums of tile length x 8.
struct DbFileHeader {
    char magic[8];  // "SWGBDB01"
    uint32_t version, alphabet;
    uint64_t n_seqs, total_residues;
    uint32_t max_len, long_threshold;
    uint64_t n_tiles, n_long_tiles, n_long, tile_bytes, residues_short, residues_long;
    uint32_t max_len_long, max_len_short;
};
constexpr char kDbMagic[8] = {'S', 'W', 'G', 'B', 'D', 'B', '0', '1'};
constexpr uint64_t kIoChunk = 64ull << 20;

bool write_all(FILE* f, const void* p, size_t n) { return n == 0 || fwrite(p, 1, n, f) == n; }
bool read_all(FILE* f, void* p, size_t n) { return n == 0 || fread(p, 1, n, f) == n; }

}  // namespace

extern "C" sw_status sw_db_save(const sw_db* db, const char* path) {
    clear_error();
    if (!db || !path) return fail(SW_ERR_INVALID_ARG, "sw_db_save: NULL argument");
    DevicePin pin(db->device);
    if (!pin.ok) return fail(SW_ERR_CUDA, "sw_db_save: cannot select device %d", db->device);
    DbFileHeader h{};
    std::memcpy(h.magic, kDbMagic, 8);
    h.version = 1;
    h.alphabet = db->alphabet;
    h.n_seqs = db->n_seqs;
    h.total_residues = db->total_residues;
    h.max_len = db->max_len;
    h.long_threshold = db->long_threshold;
    h.n_tiles = db->n_tiles;
    h.n_long_tiles = db->n_long_tiles;
    h.n_long = db->n_long;
    h.tile_bytes = db->tile_bytes;
    h.residues_short = db->residues_short;
    h.residues_long = db->residues_long;
    h.max_len_long = db->max_len_long;
    h.max_len_short = db->max_len_short;
    std::vector<uint32_t> sorted(db->n_tiles * kTileSeqs);
    cudaError_t e = cudaMemcpy(sorted.data(), db->d_sorted, sorted.size() * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "sw_db_save: sorted ids");
    FILE* f = fopen(path, "wb");
    if (!f) return fail(SW_ERR_INVALID_ARG, "sw_db_save: cannot open %s for writing", path);
    bool ok = write_all(f, &h, sizeof h) && write_all(f, db->seq_len.data(), db->n_seqs * 4) &&
              write_all(f, sorted.data(), sorted.size() * 4) &&
              write_all(f, db->tile_len_host.data(), db->n_tiles * 4);
    std::vector<uint8_t> buf;
    for (uint64_t o = 0; ok && o < db->tile_bytes; o += kIoChunk) {
        const uint64_t n = std::min(kIoChunk, db->tile_bytes - o);
        buf.resize(n);
        if ((e = cudaMemcpy(buf.data(), db->d_tile_data + o, n, cudaMemcpyDeviceToHost)) != cudaSuccess)
            break;
        ok = write_all(f, buf.data(), n);
    }
    const bool closed = fclose(f) == 0;
    if (e != cudaSuccess) return cuda_fail(e, "sw_db_save: tiles");
    if (!ok || !closed) return fail(SW_ERR_INVALID_ARG, "sw_db_save: write to %s failed", path);
    return SW_OK;
}

extern "C" sw_status sw_db_open(const char* path, const sw_db_opts* opts, sw_db** out) {
    clear_error();
    if (!out || !path) return fail(SW_ERR_INVALID_ARG, "sw_db_open: NULL argument");
    *out = nullptr;
    FILE* f = fopen(path, "rb");
    if (!f) return fail(SW_ERR_INVALID_ARG, "sw_db_open: cannot open %s", path);
    DbFileHeader h{};
    auto bad = [&](const char* why) {
        fclose(f);
        return fail(SW_ERR_INVALID_ARG, "sw_db_open: %s: %s", path, why);
    };
    if (!read_all(f, &h, sizeof h) || std::memcmp(h.magic, kDbMagic, 8) != 0 || h.version != 1)
        return bad("not a database file of this library");
    if (h.alphabet == 0 || h.alphabet > SW_MAX_ALPHABET || h.n_seqs == 0 ||
        h.n_seqs >= 0xffffffffull || h.n_tiles != (h.n_seqs + kTileSeqs - 1) / kTileSeqs ||
        h.n_long_tiles > h.n_tiles)
        return bad("inconsistent header");
    // the file must hold exactly the arrays the header announces
    const uint64_t expect = sizeof h + h.n_seqs * 4 + h.n_tiles * kTileSeqs * 4 + h.n_tiles * 4 +
                            h.tile_bytes;
    if (fseek(f, 0, SEEK_END) != 0 || (uint64_t)ftell(f) != expect ||
        fseek(f, (long)sizeof h, SEEK_SET) != 0)
        return bad("size does not match its header");
    sw_db* db = new (std::nothrow) sw_db();
    if (!db) {
        fclose(f);
        return fail(SW_ERR_OOM, "sw_db_open: host allocation failed");
    }
    auto fail_db = [&](sw_status st) {
        fclose(f);
        release(db);
        return st;
    };
    db->device = opts ? opts->device : 0;
    db->alphabet = h.alphabet;
    db->n_seqs = h.n_seqs;
    db->total_residues = h.total_residues;
    db->max_len = h.max_len;
    db->long_threshold = h.long_threshold;  // the tiles were binned with it
    db->budget = opts ? opts->device_budget : 0;
    db->flags = opts ? opts->flags : 0;
    db->n_tiles = h.n_tiles;
    db->n_long_tiles = h.n_long_tiles;
    db->n_long = h.n_long;
    db->tile_bytes = h.tile_bytes;
    db->residues_short = h.residues_short;
    db->residues_long = h.residues_long;
    db->max_len_long = h.max_len_long;
    db->max_len_short = h.max_len_short;
    db->seq_len.resize(h.n_seqs);
    std::vector<uint32_t> sorted(h.n_tiles * kTileSeqs);
    db->tile_len_host.resize(h.n_tiles);
    if (!read_all(f, db->seq_len.data(), h.n_seqs * 4) || !read_all(f, sorted.data(), sorted.size() * 4) ||
        !read_all(f, db->tile_len_host.data(), h.n_tiles * 4))
        return fail_db(fail(SW_ERR_INVALID_ARG, "sw_db_open: %s: short read", path));
    // cross-checks: every sequence once in the sorted order, tile sizes add up
    db->pos_of.assign(h.n_seqs, 0xffffffffu);
    uint64_t seen = 0, residues = 0, tile_sum = 0;
    uint32_t max_len = 0;
    for (uint64_t p = 0; p < sorted.size(); ++p) {
        const uint32_t s = sorted[p];
        if (s == 0xffffffffu) continue;
        if (s >= h.n_seqs || db->pos_of[s] != 0xffffffffu)
            return fail_db(fail(SW_ERR_INVALID_ARG, "sw_db_open: %s: bad sorted ids", path));
        db->pos_of[s] = (uint32_t)p;
        ++seen;
        if (db->seq_len[s] > db->tile_len_host[p / kTileSeqs])
            return fail_db(fail(SW_ERR_INVALID_ARG, "sw_db_open: %s: tile shorter than a sequence", path));
    }
    for (uint64_t s = 0; s < h.n_seqs; ++s) {
        residues += db->seq_len[s];
        max_len = std::max(max_len, db->seq_len[s]);
    }
    std::vector<uint64_t> tile_off(h.n_tiles);
    for (uint64_t t = 0; t < h.n_tiles; ++t) {
        tile_off[t] = tile_sum;
        tile_sum += (uint64_t)db->tile_len_host[t] * kTileSeqs;
    }
    if (seen != h.n_seqs || residues != h.total_residues || max_len != h.max_len ||
        tile_sum != h.tile_bytes)
        return fail_db(fail(SW_ERR_INVALID_ARG, "sw_db_open: %s: arrays disagree with the header", path));

    DevicePin pin(db->device);
    if (!pin.ok) return fail_db(fail(SW_ERR_CUDA, "sw_db_open: cannot select device %d", db->device));
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&db->stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreate(&db->ev_t0)) != cudaSuccess ||
        (e = cudaEventCreate(&db->ev_t1)) != cudaSuccess)
        return fail_db(cuda_fail(e, "sw_db_open: stream/event creation"));
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, db->device);
    db->nsm = prop.multiProcessorCount;
    set_block_route(db, opts ? opts->block_threshold : 0);
    sw_status st;
    if ((st = db_alloc(db, (void**)&db->d_misc, 64, "sw_db_open: counters")) ||
        (st = db_alloc(db, (void**)&db->d_tile_data, db->tile_bytes, "sw_db_open: tiles")) ||
        (st = db_alloc(db, (void**)&db->d_tile_off, h.n_tiles * 8, "sw_db_open: tile offsets")) ||
        (st = db_alloc(db, (void**)&db->d_tile_len, h.n_tiles * 4, "sw_db_open: tile lengths")) ||
        (st = db_alloc(db, (void**)&db->d_sorted, sorted.size() * 4, "sw_db_open: sorted ids")) ||
        (st = db_alloc(db, (void**)&db->d_scores, h.n_seqs * 4, "sw_db_open: score buffer")))
        return fail_db(st);
    e = cudaMemcpy(db->d_tile_off, tile_off.data(), h.n_tiles * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(db->d_tile_len, db->tile_len_host.data(), h.n_tiles * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(db->d_sorted, sorted.data(), sorted.size() * 4, cudaMemcpyHostToDevice);
    std::vector<uint8_t> buf;
    for (uint64_t o = 0; e == cudaSuccess && o < db->tile_bytes; o += kIoChunk) {
        const uint64_t n = std::min(kIoChunk, db->tile_bytes - o);
        buf.resize(n);
        if (!read_all(f, buf.data(), n))
            return fail_db(fail(SW_ERR_INVALID_ARG, "sw_db_open: %s: short read", path));
        // every byte is a residue code below the alphabet or the pad code
        for (uint64_t k = 0; k < n; ++k)
            if (buf[k] >= db->alphabet && buf[k] != kPadCode)
                return fail_db(fail(SW_ERR_INVALID_ARG, "sw_db_open: %s: bad residue code", path));
        e = cudaMemcpy(db->d_tile_data + o, buf.data(), n, cudaMemcpyHostToDevice);
    }
    fclose(f);
    f = nullptr;
    if (e != cudaSuccess) {
        st = cuda_fail(e, "sw_db_open: upload");
        release(db);
        return st;
    }
    if ((st = sw_db_prepare_search(db))) {
        release(db);
        return st;
    }
    *out = db;
    return SW_OK;
}
