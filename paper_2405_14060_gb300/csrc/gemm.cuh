// Dense pairwise contractions as batched GEMMs: operand preparation
// (permute into GEMM form, per-item power-of-two scaling, dtype conversion),
// tcgen05 tensor-core GEMM (TF32 / BF16 in, FP32 accumulate in TMEM) and a
// CUDA-core tiled GEMM (FP32 / FP64).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include <vector>

#include "kernels.cuh"

namespace tn {

enum ElemType { E_F64 = 0, E_F32 = 1, E_BF16 = 2 };

// Permute a strided tensor into a dense layout (optionally with padded
// innermost stride), scaling each batch item by 2^-e(max) and converting.
//   logical dims (slowest first): sz[d]; input stride sin[d]; output stride sout[d]
//   beta_dim: the dimension that indexes batch items for the scale (-1: none)
//   mxo (optional): record the per-item maximum of the output (beta from beta_dim)
// Tiled form of a permutation (chosen on the host when it pays): every dim
// whose input or output stride is below 32 elements goes into one tile of
// tn <= 4096 entries staged in shared memory, so that loads run along the
// input's contiguous runs and stores along the output's; the other dims
// enumerate the tiles.  Device table ttab (16-byte aligned): input offsets
// [tn] (input order), output offsets [tn] (output order), and for each
// output-order entry its shared-memory slot as 16-bit integers [tn].  The
// slot of input-order entry e follows the layout `swz` (pt_slot), chosen on
// the host as the one with the fewest shared-memory wavefronts for the
// tile's read pattern.
constexpr int PT_MAXN = 4096;

// Shared-memory slot of input-order tile entry e: layout 0 pads every run of
// 32 entries by 4; layouts 1-3 permute the 16-byte groups inside each run of
// 32 entries by an XOR with a hash of the run index.  All keep 16-byte
// groups whole, so 16-byte asynchronous copies stay aligned.
constexpr int PT_NSWZ = 4;
template <int ESZ>
__host__ __device__ __forceinline__ int pt_slot(int e, int swz) {
    constexpr int GI = 16 / ESZ;   // entries per 16-byte group
    if (swz == 0) return e + 4 * (e >> 5);
    const int r = e >> 5, w = e & 31;
    const int h = (swz == 1 ? r ^ (r >> 3) : swz == 2 ? r ^ ((r >> 3) << 1) : r) & 7;
    return (r << 5) + ((w / GI) ^ h) * GI + (w % GI);
}

// Shared-memory entries of one tile buffer of n entries in layout swz.
__host__ __device__ __forceinline__ int pt_nbuf(int n, int swz) {
    return swz == 0 ? n + 4 * (n >> 5) + 4 : (n + 31) & ~31;
}

struct PTile {
    int tn;                          // 0: not tiled
    int swz;                         // shared-memory layout of a tile (pt_slot)
    int nbuf;                        // shared-memory entries per tile buffer
    int nrest, rest_beta;            // rest dims, index of the batch dim among them (-1)
    int32_t rsz[MAXD], rsh[MAXD];    // rest sizes, log2 (-1: not a power of two)
    int64_t rin[MAXD], rout[MAXD];
    int64_t ntiles;
    int vec;                         // outputs per 16-byte store (0: one at a time)
    int vin;                         // inputs per 16-byte copy (0: one at a time)
    const int32_t *ttab;
};

struct PDesc {
    int nd;
    int pow2;
    int beta_dim;
    int in_type, out_type;      // ElemType
    int64_t total;
    int32_t sz[MAXD], sh[MAXD];
    int64_t sin[MAXD], sout[MAXD];
    const void *in;
    void *out;
    const unsigned long long *mxi;   // scale source (NULL: no scaling)
    int mxi_bs;                      // 1: per item
    unsigned long long *mxo;
    PTile tl;
};

// Choose the tiled form for p when it pays (host): fills p.tl (but for the
// device table pointer) and the table; leaves p.tl.tn = 0 otherwise.
void plan_permute_tiles(PDesc &p, std::vector<int32_t> &tab);

// D[b][r][c] = sum_k X[b][r][k] * Y[b][c][k]   (X, Y K-major, D row-major FP32/FP64)
struct GDesc {
    int64_t R, C, K, batch;
    int64_t ldx, ldy, ldd;          // elements
    int64_t bsx, bsy, bsd;          // elements
    int xtype;                      // ElemType of X and Y
    const void *X, *Y;
    void *D;
    unsigned long long *mxd;        // per-item max of D (NULL: none)
    const unsigned long long *mxsx; // X read in place: D is scaled by 2^-e of this maximum
    int64_t beta_div_batch;         // item = b / beta_div_batch (if > 0)
    int64_t beta_div_row;           // else item = r / beta_div_row (if > 0), else 0
};

void launch_permute(const PDesc &p, cudaStream_t st);
// Returns false if the tensor-core path cannot take this problem.
bool tc_gemm_supported(const GDesc &g);
cudaError_t launch_tc_gemm(const GDesc &g, int *err_flag, cudaStream_t st);
void launch_simt_gemm(const GDesc &g, cudaStream_t st);

}  // namespace tn
