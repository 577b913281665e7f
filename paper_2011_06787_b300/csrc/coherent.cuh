// Sky-table object and coherent-scan kernel arguments (internal).
#pragma once

#include <cstring>
#include <vector>

#include "common.cuh"

namespace spiir {

constexpr int kCohThreads = 256;                 // threads per block
constexpr int kCohQ = 2;                         // output samples per thread
constexpr int kCohMaxHalo = 1024;                // largest |Delta_I(p)| accepted
constexpr int kCohSmemTableLimit = 112 * 1024;   // table + SNR tile kept in shared memory below this

struct CohArgs {
    const float2 *snr;   // [T][n_det][pitch], entry H + k is output sample k
    int64_t pitch;
    int n_templates;
    int64_t n;
    int H;
    int n_pix;
    const void *table;   // [n_pix] entries: U_s columns and offsets H + Delta_I
    const float *u_null; // [n_pix][n_det][n_det - 2]
    float *max_stat;
    int32_t *argmax;
    float *null_stat;
    float *skymap;       // NULL or [T][n_pix][n]
    size_t tab_bytes;    // bytes of the table staged in shared memory (0: read from global)
};

}  // namespace spiir

struct spiir_sky_s {
    int n_det = 0, n_pix = 0, halo = 0;
    std::vector<unsigned char> h_table;
    size_t table_bytes = 0;
    void *table = nullptr;
    float *u_null = nullptr;
};

namespace spiir {
int coherent_scan(spiir_sky_s *sky, const float2 *snr, int64_t pitch, int T, int64_t n, float *max_stat,
                  int32_t *argmax, float *null_stat, float *skymap, cudaStream_t stream);
}
