// HBM-bound pairwise contractions that stream their large operands once.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace tn {

constexpr int AMAX = 32;   // summed / new label combinations handled per thread

// Absorb: Y[t, r] = (+)_s X[r, s] (x) W[r_w, s, t]
//   r: positions shared by X and Y (one thread each, Y's order)
//   s: labels summed here (in X and/or W), t: labels new to Y (from W)
// X is streamed once; W is small and read through L1.
struct ADesc {
    int nrd, pow2r;
    int nin_d;                        // the last nin_d R dims are "inner" (32-bit offsets)
    int64_t nin, nouter;              // inner / outer position counts per item
    int32_t rsz[MAXD], rsh[MAXD];
    int64_t rsx[MAXD], rsy[MAXD], rsw[MAXD];
    int64_t nr;                       // positions per batch item
    int ns, nt;
    int32_t xoff[AMAX], wso[AMAX];    // per summed combination (offsets within an item)
    int32_t yoff[AMAX], wto[AMAX];    // per new combination
    int nbeta;
    int64_t bsx, bsw, bsy;
    const void *X, *W;
    void *Y;
    const unsigned long long *mxx, *mxw;
    int mxx_bs, mxw_bs;
    unsigned long long *mxy;
    int32_t *argmax;                  // max-plus: flat summed index per output
    const int32_t *tab;               // inner offsets: X [nin], Y [nin], W [nin], then the
                                      // shared-label index [nin] and the W offset of every
                                      // shared-label combination [nsh] (device)
    int nsh;                          // combinations of the labels W shares with X and Y
    int32_t rshc[MAXD];               // per R dim: stride in that combination index (0: not in W)
    int bps;                          // blocks per SM of the launch (0: the kernel's default)
    // dense kernel (dense_impl.cuh): chunk tables of X's and Y's tiles in tab
    // (positions; used when cx / cy are set)
    int cx, cy;
    int32_t cxo, cyo;
};

// Reduce: O[g, s, t] = sum_m X[g, m, s] Z[g, m, t]
//   g: groups (labels in X, Z and O, plus the batch item) -> blockIdx.y
//   m: summed positions (labels absent from O) streamed by the block
//   s: labels of X kept in O, t: labels of Z kept in O  (ns * nt <= 64)
struct RDesc {
    int ngd, nmd, pow2m;
    int nin_d;                        // the last nin_d summed dims are "inner" (offset table)
    int64_t nin, nouter;
    int32_t gsz[MAXD];
    int64_t gsx[MAXD], gsz2[MAXD], gso[MAXD];
    int32_t msz[MAXD], msh[MAXD];
    int64_t msx[MAXD], msz2[MAXD];
    int64_t ng, nm;                   // groups per item, summed positions
    int ns, nt;
    int64_t xoff[AMAX], oso[AMAX];
    int64_t zoff[AMAX], oto[AMAX];
    int nbeta;
    int64_t bsx, bsz, bso;
    const void *X, *Z;
    void *O;
    const unsigned long long *mxx, *mxz;
    int mxx_bs, mxz_bs;
    unsigned long long *mxo;
    const int32_t *tab;               // inner offsets: X [nin], Z [nin] (device)
    unsigned int *cnt;                // per group: blocks done (zero between launches)
    // dense kernel (dense_impl.cuh): chunk tables of X's and Z's tiles in tab
    int cx, cz;
    int32_t cxo, czo;
};

template <typename T>
void launch_absorb(const ADesc &d, int semiring, cudaStream_t st);
size_t reduce_scratch_bytes(const RDesc &d, int elem_bytes);
template <typename T>
void launch_reduce(const RDesc &d, void *scratch, cudaStream_t st);
int reduce_launches(const RDesc &d);
// Does the reduce run as k_reduce_vec (16-byte vector loads)?
bool reduce_vector_form(const RDesc &d, int elem_bytes);
// Plan trace: the dense kernels' load / store modes (-1: not the dense form).
void absorb_dense_describe(const ADesc &d, int &xm, int &ym);
bool absorb_dense_form_host(const ADesc &d);
int reduce_dense_describe(const RDesc &d);

}  // namespace tn
