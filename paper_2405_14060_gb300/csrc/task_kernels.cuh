// Task-level kernels (leaves, log Z, marginals, backtracking, sampling).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace tn {

enum LeafKind { LEAF_FACTOR = 0, LEAF_UNITY = 1, LEAF_EXTERNAL = 2 };

constexpr int LEAF_D = 16;   // scope size of a factor leaf that can be sliced

struct LeafRec {
    int kind;
    int var;              // unity: variable id
    int beta;             // unity: carries the batch label
    int slice_of_var;     // unity: index of the variable among the sliced ones, or -1
    int64_t src;          // factor: table offset; external: device address of the data
    int64_t size;         // entries per item
    int64_t dst;          // element offset of the leaf in the arena
    int64_t mx;           // index of its first maximum slot
    const double *sigma;  // external: log2 scale of the data (device), or NULL
    // factor leaf with sliced labels (nkd >= 0): entry i of the leaf is the
    // table entry at sum_j digit_j(i) * kst[j] + sum_j slice_val[sidx[j]] * sst[j]
    int nkd, nsd;
    int32_t ksz[LEAF_D], sidx[LEAF_D];
    int64_t kst[LEAF_D], sst[LEAF_D];
};

struct MargRec {
    int64_t fwd, adj;     // element offsets of u_v and of its adjoint
    int64_t moff;         // offset of variable v's block in a marginal row
    int card, fbeta, abeta, sliced;   // sliced: marginal filled by the slice combination
};

struct GradRec {
    int64_t fwd, adj, size, goff;
    int abeta, pad;
};

template <typename T>
void launch_leaves(const LeafRec *recs, int nrec, const double *tables, const int *card,
                   int nvars, const int32_t *evid, int nbeta, int log_mode, T *base,
                   unsigned long long *mx, const int *flags, const int32_t *slice_val,
                   cudaStream_t st);
// Slice combination (sum over slice assignments, Sec. "Tensor networks":
// slicing fixes variables; the contraction is the sum over their values):
// running log-sum-exp of log Z and Z-weighted marginals, per batch item.
void launch_slice_init(int nbeta, int64_t nm, double *M, double *S, double *A, cudaStream_t st);
void launch_slice_acc(int nbeta, const double *logz, const double *marg, int64_t nm,
                      const int32_t *slice_val, int nsl, const int32_t *sl_var,
                      const int64_t *sl_moff, const int32_t *sl_card, double *M, double *S,
                      double *A, cudaStream_t st);
void launch_slice_fin(int nbeta, int64_t nm, const double *M, const double *S, const double *A,
                      double *logz, double *marg, cudaStream_t st);
template <typename T>
void launch_logz(int nbeta, const T *root, int root_beta, const unsigned long long *mx,
                 const int64_t *exps, int nexp, double *logz, double *sigma_out, int maxplus,
                 cudaStream_t st);
template <typename T>
void launch_fill_one(T *p, int64_t n, unsigned long long *mx, cudaStream_t st);
template <typename T>
void launch_marginals(const MargRec *recs, int nvars, int nbeta, const T *fbase, const T *abase,
                      double *marg, int64_t mstride, cudaStream_t st);
template <typename T>
void launch_factor_grads(const GradRec *recs, int nrec, int nbeta, const T *fbase,
                         const T *abase, double *grad, int64_t gstride, cudaStream_t st);
void launch_backtrack(const int64_t *meta, int nnodes, const int32_t *argmax, int nbeta,
                      int nvars, int32_t *assign, cudaStream_t st);
template <typename T>
void launch_sample(const int64_t *meta, int nnodes, const T *base, const double *cdf,
                   const int32_t *evid, int nvars, int64_t nsamp, uint64_t seed, int8_t *out,
                   cudaStream_t st);
template <typename T>
void launch_cdf_rows(const CDesc &d, int64_t rows, double *cdf, cudaStream_t st);

}  // namespace tn
