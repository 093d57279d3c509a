// Learned far field, data path (rp_learned_data.cu): structures and launchers.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "rp_internal.h"
#include "rp_learned.h"

namespace rp {

constexpr int kLGauss = 3;        // Gaussians per training history
constexpr int kLHistT = 64;       // amplitude samples per training history
constexpr int kLSampGroup = 8;    // label samples per block of the label kernel

// Moments of one source slice about its box centre, into out[slot % out_depth].
// The slice is rho / J if set, else the pushed slice of domain `dom`.
struct MomentJob {
    const float *rho, *J;    // [N] and [3][N]
    int dom;
    int nx, ny, nz;
    double h;
    double ox, oy, oz;       // origin - centre
    double *part;            // [4][nz][10] scratch
    float *out;              // [out_depth][4][10]
    int out_depth;
};

// A (source -> target) pair of the learned path, or one training history.
struct LPair {
    float R[9];              // canonical frame, rows
    double tau_c;            // centre-to-centre delay in steps
    float Rc;                // centre-to-centre distance
    const float *mom;        // moment history [mdepth][4][10] (ring or array)
    int mdepth;
    float yscale;            // weight of the network's output (0: the linear skip alone)
    const float *P;          // [64][r] canonical -> target-node interpolation, transposed
    float Ra[kLOut];         // distances from c_s to the canonical nodes
};

// One network sample: pair index and the window centre time (steps).
struct FeatRow {
    int pair;
    double tc;
};

// A far target with learned pairs [p0, p1) (pairs sorted by target).
struct LTarget {
    float *cring;
    int depth, r;
    int p0, p1;
    int overwrite;           // no low-rank pairs: the slot is set, not added to
    int pad_;
};

// One synthetic training history: Gaussians on the source grid (coordinates
// relative to the source origin), amplitude tables, and the geometry of the
// canonical nodes relative to the source centre.
struct TrainHist {
    float cx[kLGauss], cy[kLGauss], cz[kLGauss], sigma[kLGauss];
    float amp[kLGauss][kLHistT];    // A_g(t_j)
    float damp[kLGauss][kLHistT];   // dA_g/dt (t_j) / (4 pi)
    float csx, csy, csz;            // source centre relative to its origin
    float R[9];                     // canonical frame
    float D[kLOut][3];              // canonical node - source centre (world axes)
    float Dn[kLOut];                // |D|
    float base[kLOut];              // retarded time index (at the source centre) of sample 0
};

cudaError_t launch_moments(const MomentJob *d_jobs, int njobs, int max_nz, long long slot, const IoPtrs *in,
                           cudaStream_t s);
cudaError_t launch_features(const LPair *d_pairs, const FeatRow *d_rows, int nrows, long long step, __half *X16,
                            float *Xf, float *nu, cudaStream_t s);
cudaError_t launch_train_basis(const TrainHist *d_hist, int nhist, const int n[3], float h, float *B, cudaStream_t s);
cudaError_t launch_train_moments(const TrainHist *d_hist, int nhist, const float *Mb, int T, float *mom,
                                 cudaStream_t s);
cudaError_t launch_train_labels(const TrainHist *d_hist, int nhist, const float *B, const int n[3], float h,
                                int samples, double cdt, float *labels, cudaStream_t s);
cudaError_t launch_label_rows(const TrainHist *d_hist, int nhist, const float *labels, const float *nu, int samples,
                              float *Y, cudaStream_t s);
// c += re-interpolated nu * (pair.yscale * Y + Ylin) / R_a (network output
// plus linear skip), summed over each target's pairs in pair order; pair_r[p]
// is the pair's target node count, contrib scratch [npairs][64][4].
cudaError_t launch_learned_out(const LTarget *d_tgts, int ntgt, const LPair *d_pairs, int npairs, const int *d_pair_r,
                               const float *Y, const float *Ylin, const float *nu, float *contrib, long long step,
                               cudaStream_t s);

}  // namespace rp
