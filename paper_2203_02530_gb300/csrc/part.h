// Plan object behind the opaque spmv_part handle (include/spmv.h).
#pragma once

#include "internal.h"
#include "../../include/spmv.h"

#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdint>
#include <map>
#include <string>
#include <utility>
#include <vector>

namespace spmvk {

// Raised inside the library, turned into a status at the ABI.
struct Fail {
    int code;
    std::string msg;
};
[[noreturn]] void fail(int code, const char* fmt, ...);
void check_cuda(cudaError_t e, const char* what);
void set_last_error(const std::string& msg);   // message of spmv_last_error()

// Device allocation owned by a plan.  Every array is padded by kPad bytes
// (zero-filled) so that the 16-byte-rounded bulk copies and 128-bit vector
// loads near the end of an array stay inside the allocation.
constexpr size_t kPad = 256;

struct DevArray {
    void* p = nullptr;
    size_t bytes = 0;   // payload bytes (without padding)
};

struct GraphRec {
    cudaGraphExec_t exec = nullptr;
    const double* x = nullptr;
    double* y = nullptr;
};

}  // namespace spmvk

struct spmv_part {
    int device = 0;
    int num_sms = 0;
    int64_t n = 0;
    int P = 1;
    int gran = SPMV_COARSE;
    std::vector<int64_t> bounds;      // P+1 row bounds r_p

    // sizes
    int64_t nnz = 0, nnz_l = 0, nnz_r = 0, n_send = 0, n_rr = 0;
    std::vector<int64_t> halo_off;    // P+1 destination offsets in the send buffer
    std::vector<int64_t> seg_off;     // P*P+1 segment (dst p, src q) offsets
    std::vector<int64_t> rr_off;      // P+1 offsets into the remote-row list per rank
    std::vector<int64_t> pack_off;    // P+1 offsets into pack_pos per source rank

    // device arrays
    // A_L of every rank as one CSR over the n global rows with columns
    // rebased to the owning block (x_L = x + r_p).
    int32_t* l_ptr = nullptr;         // n+1
    int32_t* l_col = nullptr;
    double* l_val = nullptr;
    // A_R compressed to the rows that have remote entries
    int32_t* rr_row = nullptr;        // n_rr global row ids
    int32_t* rr_ptr = nullptr;        // n_rr+1
    int32_t* r_col = nullptr;         // positions in the receive buffer
    double* r_val = nullptr;
    int32_t* send_idx = nullptr;      // n_send global x indices
    int32_t* pack_pos = nullptr;      // n_send send slots grouped by source rank
    double* sendbuf = nullptr;
    double* recvbuf = nullptr;
    int* err = nullptr;               // device error word
    double* io_x = nullptr;           // plan-owned x / y for the host-buffer path
    double* io_y = nullptr;
    double* io_x2 = nullptr;          // the second x / y pair of the streamed host path
    double* io_y2 = nullptr;
    std::vector<cudaEvent_t> io_ev;   // 3P+1: x block p arrived; LOCAL p done; REMOTE p done; exchange done;
                                      // then x free and y free per pair of the streamed host path
    cudaStream_t io_out = nullptr;    // the host path's copies of y out
    cudaStream_t io_alt = nullptr;    // the host path's second stream for LOCAL / REMOTE products
    cudaStream_t io_aux = nullptr;    // the host path's stream for pack and exchange
    // per rank: the longest run [a, b) of rows without remote entries (final
    // after the rank's LOCAL product; the host path copies it out early)
    std::vector<std::pair<int64_t, int64_t>> io_free;

    // tiles (thread-per-row and vector kernels)
    spmvk::TileGeom geom{};
    spmvk::Tile* ltiles = nullptr;
    spmvk::Tile* rtiles = nullptr;
    std::vector<int64_t> ltile_off;   // P+1
    std::vector<int64_t> rtile_off;   // P+1
    // fixed 256-row blocks (vector and pair kernels): independent of the
    // tile geometry so their passes of 256 / lanes rows are always full
    spmvk::Tile* lblocks = nullptr;
    spmvk::Tile* rblocks = nullptr;
    std::vector<int64_t> lblock_off;  // P+1
    std::vector<int64_t> rblock_off;  // P+1
    // 32-row tiles of the warp-pipeline kernel (built on first use)
    spmvk::Tile* lwtiles = nullptr;
    spmvk::Tile* rwtiles = nullptr;
    std::vector<int64_t> lwtile_off;  // P+1
    std::vector<int64_t> rwtile_off;  // P+1
    int wtile_cap = 0;
    // merge-path tiles (built on first use of the merge variant)
    spmvk::MergeTile* lmtiles = nullptr;
    spmvk::MergeTile* rmtiles = nullptr;
    spmvk::Carry* lcarry = nullptr;
    spmvk::Carry* rcarry = nullptr;
    std::vector<int64_t> lmtile_off;  // P+1
    std::vector<int64_t> rmtile_off;  // P+1

    // sliced-ELL copies of A_L [0] and A_R [1] (built on first use of that
    // variant): slices and long rows per rank, row order per position
    struct SellPart {
        spmvk::SellSlice* slices = nullptr;
        spmvk::SellLong* longs = nullptr;
        double* val = nullptr;
        int32_t* col = nullptr;
        uint8_t* len = nullptr;
        int32_t* perm = nullptr;          // nullptr: every rank in natural order
        int32_t* ypos = nullptr;          // REMOTE, sorted: y row of each position (perm, then the row map)
        int16_t* col16 = nullptr;         // column - row deltas (LOCAL only), once built
        double* long_part = nullptr;      // partial sums of cut long rows
        int* long_cnt = nullptr;          // pieces done per cut long row
        std::vector<int32_t> h_slice_len; // per slice: its longest row's entries
        std::vector<int32_t> h_long_len;  // per long-row piece: its entries
        // balanced CTA ranges per launch site (rank p, or P for all ranks)
        // and grid: key site << 32 | grid
        std::map<int64_t, int32_t*> cta_split;
        int delta_state = 0;              // 0 not checked, 1 built, -1 some delta needs > 16 bits
        // with the CSR released: the long rows' entries, piece after piece
        // (the pieces' k0/k1 then index these), and each piece's CSR start
        double* long_val = nullptr;
        int32_t* long_col = nullptr;
        std::vector<int32_t> h_long_csr_k0;
        int64_t entries = 0;              // padded slots
        std::vector<int64_t> slice_off;   // P+1
        std::vector<int64_t> long_off;    // P+1
        std::vector<char> sorted;         // per rank
    } sell[2];
    bool sell_built = false;
    bool csr_released = false;        // l_col/l_val/r_col/r_val freed (spmv_part_release_csr)
    int64_t sell_entries = 0;         // padded entries, local + remote

    // product variant of the LOCAL [0] and REMOTE [1] operations
    int variant[2] = {SPMV_VARIANT_TILE, SPMV_VARIANT_TILE};
    int vparam[2] = {0, 0};

    // halo segments (destination p, source q, send slots [a, b)), nonempty,
    // destination-major: the pack/copy ops of the per-segment granularity
    struct Seg {
        int p, q;
        int64_t a, b;
    };
    std::vector<Seg> segs;

    // DAG of the operations
    int n_ops = 0;
    std::vector<std::pair<int, int>> edges;
    std::vector<std::vector<int>> preds;

    // schedule runtime
    std::vector<cudaEvent_t> op_ev;   // one per op
    std::vector<cudaEvent_t> join_ev; // one per stream slot (grown on demand)
    cudaEvent_t fork_ev = nullptr;
    std::map<int64_t, spmvk::GraphRec> graphs;
    // captured deferred remote products: (its kernel's node, the node of the
    // kernel before it on its stream), for the edge check after capture
    std::vector<std::pair<cudaGraphNode_t, cudaGraphNode_t>> deferred_nodes;
    int64_t next_graph = 1;
    int64_t last_records = 0, last_waits = 0, last_launches = 0, last_deferred = 0;
    int cur_pdl = 0;                  // programmatic-launch flags of the op being issued
    bool dry_run = false;             // ops count the kernels they would launch, and launch none

    std::vector<spmvk::DevArray> allocs;   // everything to free
    size_t device_bytes = 0;
};

namespace spmvk {
void validate_csr(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, const double* vals, int P);
void build_plan(spmv_part* pt, int64_t n, const int64_t* row_ptr, const int32_t* col_idx,
                const double* vals);
void build_tiles(spmv_part* pt, const TileGeom& g);
void build_merge_tiles(spmv_part* pt);
void build_warp_tiles(spmv_part* pt, int cap);
void build_sell(spmv_part* pt);
bool build_sell_delta16(spmv_part* pt);
void build_sell_split(spmv_part* pt, int part_idx, int param);
void release_csr(spmv_part* pt);
void restore_csr(spmv_part* pt);
const int32_t* sell_split(const spmv_part* pt, int part_idx, int site, int grid);
void* dev_alloc(spmv_part* pt, size_t bytes);
void free_plan(spmv_part* pt);
}  // namespace spmvk
