// Autotuner: measured kernel shapes for one database on this GPU.
//
// For every kernel mode (one query against database pairs with the int8
// query profile, two queries per lane pair, int32, one query against pairs
// with the score-profile ring) and every rows-per-lane choice R, the tuner times the
// search kernel on a sample of the database's shorter sequences with a query
// whose length fills whole passes, and records the device time per query row
// and database residue. The search paths then pick R per query (or batch) by
// minimising padded rows x measured cost instead of the built-in estimate.
// The same table gives the int16 / int32 speed ratio and with it the fraction
// of saturating pairs above which a search would be cheaper in int32 (the
// 16/32-bit cutover). Results can be cached in a small JSON file keyed by the
// GPU name and SM count.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "sw.h"
#include "sw_db.h"
#include "sw_internal.h"

using namespace swgb;

namespace {

const int kR[kTuneR] = {8, 12, 16, 20, 24};

std::string gpu_key(int device) {
    cudaDeviceProp p;
    cudaGetDeviceProperties(&p, device);
    char buf[320];
    snprintf(buf, sizeof buf, "%s|sm=%d", p.name, p.multiProcessorCount);
    return buf;
}

bool load_cache(const char* path, const std::string& key, sw_tuning* t) {
    if (!path) return false;
    FILE* f = fopen(path, "r");
    if (!f) return false;
    std::string s;
    char buf[4096];
    size_t n;
    while ((n = fread(buf, 1, sizeof buf, f)) > 0) s.append(buf, n);
    fclose(f);
    const std::string want = "\"gpu\": \"" + key + "\"";
    if (s.find(want) == std::string::npos) return false;
    auto read_row = [&](const char* name, double* out, int cnt) {
        const size_t p = s.find(std::string("\"") + name + "\"");
        if (p == std::string::npos) return false;
        size_t q = s.find('[', p);
        for (int i = 0; i < cnt; ++i) {
            char* end = nullptr;
            out[i] = strtod(s.c_str() + q + 1, &end);
            q = end - s.c_str();
            if (i + 1 < cnt) q = s.find(',', q);
        }
        return true;
    };
    return read_row("pair_db", t->ns_per_row_residue[0], kTuneR) &&
           read_row("query_pair", t->ns_per_row_residue[1], kTuneR) &&
           read_row("int32", t->ns_per_row_residue[2], kTuneR) &&
           read_row("pair_ring", t->ns_per_row_residue[3], kTuneR);
}

void save_cache(const char* path, const std::string& key, const sw_tuning* t) {
    if (!path) return;
    FILE* f = fopen(path, "w");
    if (!f) return;
    fprintf(f, "{\n  \"gpu\": \"%s\",\n  \"rows_per_lane\": [8, 12, 16, 20, 24],\n", key.c_str());
    const char* names[kModes] = {"pair_db", "query_pair", "int32", "pair_ring"};
    for (int m = 0; m < kModes; ++m) {
        fprintf(f, "  \"%s\": [", names[m]);
        for (int i = 0; i < kTuneR; ++i)
            fprintf(f, "%.6g%s", t->ns_per_row_residue[m][i], i + 1 < kTuneR ? ", " : "");
        fprintf(f, "]%s\n", m + 1 < kModes ? "," : "");
    }
    fprintf(f, "}\n");
    fclose(f);
}

}  // namespace

extern "C" sw_status sw_db_autotune(sw_db* db, const int8_t* matrix, int32_t alpha, int32_t beta,
                                    const char* cache_path, sw_tuning* out) {
    clear_error();
    if (!db || !matrix) return fail(SW_ERR_INVALID_ARG, "sw_db_autotune: NULL argument");
    cudaSetDevice(db->device);
    sw_tuning t{};
    const std::string key = gpu_key(db->device);
    bool cached = load_cache(cache_path, key, &t);
    cudaError_t e;
    if (!cached) {
        // sample: consecutive sequences of the shorter bin centred on its residue-weighted
        // median (the lengths that carry most of the work), as many as make whole rounds of
        // the persistent grid for every mode (4 rounds of 64-sequence chunks for the modes
        // that pack two sequences, 8 of 32-sequence chunks for the others): a partial last
        // round would weigh each mode's timing by a different share of idle SMs
        const uint64_t short_units = (db->n_tiles - db->n_long_tiles) * kTileSeqs;
        const uint64_t rounds = (uint64_t)db->grid_short * 2 * wavefront_short_units_per_chunk() * 4;
        const uint64_t sample = std::min<uint64_t>(short_units, rounds);
        uint64_t centre = db->n_long_tiles;  // tile at the residue median of the short bin
        {
            uint64_t total = 0, acc = 0;
            for (uint64_t u = db->n_long_tiles; u < db->n_tiles; ++u) total += db->tile_len_host[u];
            for (uint64_t u = db->n_long_tiles; u < db->n_tiles; ++u) {
                acc += db->tile_len_host[u];
                if (2 * acc >= total) { centre = u; break; }
            }
        }
        const uint64_t lo = db->n_long_tiles * kTileSeqs;
        uint64_t first = centre * kTileSeqs > lo + sample / 2 ? centre * kTileSeqs - sample / 2 : lo;
        if (first + sample > lo + short_units) first = lo + short_units - sample;
        first &= ~(uint64_t)(kTileSeqs - 1);  // whole tiles, whole pairs
        uint64_t residues = 0;  // padded residues in the sample
        for (uint64_t u = first / kTileSeqs; u < (first + sample + kTileSeqs - 1) / kTileSeqs; ++u)
            residues += (uint64_t)db->tile_len_host[u] * kTileSeqs;
        if (sample == 0 || residues == 0)
            return fail(SW_ERR_INVALID_ARG, "sw_db_autotune: database too small to sample");
        const size_t mbytes = (size_t)db->alphabet * db->alphabet;
        std::vector<uint8_t> q(8 * 24 * 4 * 2);
        for (size_t i = 0; i < q.size(); ++i) q[i] = (uint8_t)((i * 7 + 3) % db->alphabet);
        sw_status st;
        if ((st = ensure(db, db->b_queries, q.size(), "tune query")) ||
            (st = ensure(db, db->b_pairs, sizeof(QueryPair), "tune pair")) ||
            (st = ensure(db, db->b_scores, (size_t)2 * db->n_seqs * 4, "tune scores")) ||
            (st = ensure(db, db->b_flags, (size_t)db->n_seqs * sizeof(uint2), "tune flags")))
            return st;
        if ((e = cudaMemcpyAsync(db->b_queries.p, q.data(), q.size(), cudaMemcpyHostToDevice,
                                 db->stream)) != cudaSuccess ||
            (e = cudaMemcpyAsync(db->d_matrix, matrix, mbytes, cudaMemcpyHostToDevice,
                                 db->stream)) != cudaSuccess)
            return cuda_fail(e, "sw_db_autotune: upload");
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        for (int mode = 0; mode < kModes; ++mode) {
            for (int i = 0; i < kTuneR; ++i) {
                const int R = kR[i];
                const KernelChoice kc{(KernelChoice::Mode)mode, R};
                t.ns_per_row_residue[mode][i] = 0;
                if (!wavefront_supported(kc)) continue;
                const uint32_t qlen = 8u * R * 4;  // four whole passes
                WavefrontArgs a{};
                a.dbg = db->d_counters + kDebugWord;
                a.tile_data = db->d_tile_data;
                a.tile_off = db->d_tile_off;
                a.tile_len = db->d_tile_len;
                a.sorted_ids = db->d_sorted;
                a.matrix = db->d_matrix;
                a.alphabet = db->alphabet;
                a.alpha = alpha;
                a.beta = beta;
                a.scores = (int32_t*)db->b_scores.p;
                a.score_stride = db->n_seqs;
                a.flag_list = (uint2*)db->b_flags.p;
                a.flag_cap = (uint32_t)db->n_seqs;
                a.flag_count = db->d_counters + 3;
                a.work_counter = db->d_counters + 0;
                a.query = (const uint8_t*)db->b_queries.p;
                a.qlen = qlen;
                a.bin[1].boundary = db->d_bnd_short;
                a.bin[1].bstride = db->bstride_short;
                const uint64_t per = units_per_tile(kc) == kTilePairs ? 2 : 1;
                a.bin[1].first_unit = first / per;
                a.bin[1].n_units = sample / per;
                if (mode == KernelChoice::kQueryPair) {
                    QueryPair p{};
                    p.off_a = 0;
                    p.off_b = qlen;
                    p.len_a = p.len_b = qlen;
                    p.q_a = 0;
                    p.q_b = 1;
                    cudaMemcpyAsync(db->b_pairs.p, &p, sizeof p, cudaMemcpyHostToDevice, db->stream);
                    a.pairs = (const QueryPair*)db->b_pairs.p;
                    a.n_pairs = 1;
                }
                const int occ = std::max(1, wavefront_occupancy(kc, nullptr));
                const int grid = std::max(1, std::min(db->grid_short, db->nsm * occ));
                float best = 1e30f;
                for (int rep = 0; rep < 5; ++rep) {
                    cudaMemsetAsync(db->d_counters, 0, 64, db->stream);
                    cudaEventRecord(e0, db->stream);
                    if ((e = launch_wavefront(kc, a, grid, db->stream)) != cudaSuccess) break;
                    cudaEventRecord(e1, db->stream);
                    if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
                    float ms = 0;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (rep > 0) best = std::min(best, ms);
                }
                if (e != cudaSuccess) {
                    cudaEventDestroy(e0);
                    cudaEventDestroy(e1);
                    return cuda_fail(e, "sw_db_autotune: timing launch");
                }
                // rows x residues of useful cells (two queries share a launch in query-pair mode)
                const double rowres = (double)qlen * residues * (mode == KernelChoice::kQueryPair ? 2 : 1);
                t.ns_per_row_residue[mode][i] = best * 1e6 / rowres;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        save_cache(cache_path, key, &t);
    }
    // the 16/32-bit cutover: int32 wins when more than this fraction of pairs would be
    // rescored (rescoring redoes a pair in int32 after its 16-bit pass)
    // (16-bit: the faster of the two single-query modes at R = 16)
    double c16 = t.ns_per_row_residue[0][2];
    const double ring16 = t.ns_per_row_residue[3][2];
    if (ring16 > 0 && (c16 <= 0 || ring16 < c16)) c16 = ring16;
    const double c32 = t.ns_per_row_residue[2][2];
    t.int32_over_int16 = c16 > 0 ? c32 / c16 : 0;
    t.cutover_fraction = c32 > 0 ? std::max(0.0, 1.0 - c16 / c32) : 0;
    t.from_cache = cached ? 1 : 0;
    for (int m = 0; m < kModes; ++m) {
        int bi = 0;
        for (int i = 0; i < kTuneR; ++i)
            if (t.ns_per_row_residue[m][i] > 0 &&
                (t.ns_per_row_residue[m][bi] <= 0 ||
                 t.ns_per_row_residue[m][i] < t.ns_per_row_residue[m][bi]))
                bi = i;
        t.fastest_R[m] = kR[bi];
    }
    db->tuning = t;
    db->tuned = true;
    if (out) *out = t;
    return SW_OK;
}
