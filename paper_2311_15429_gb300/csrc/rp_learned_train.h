// Learned far field, host side (rp_learned_train.cu).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "rp_learned.h"
#include "rp_learned_data.h"

namespace rp {

// Geometry of the (source box -> target box) pairs of a data set: a fixed
// direction and distance, or (random) uniform directions and log-uniform
// distances in [R_lo, R_hi].
struct LGeom {
    int n_s[3];
    double h_s;
    double Lt[3];          // target box extents (the canonical node cube has half-width |Lt| / 2)
    bool random;
    double dir[3], Rc;     // fixed geometry
    double R_lo, R_hi;     // random geometry
    // fixed geometry only: the label nodes, as world-axis offsets from the
    // target centre (kLOut of them); null: the canonical nodes
    const double (*label_nodes)[3] = nullptr;
};

// Rotation whose first row is n / |n| (see rp_learned_data.cu).
void canonical_frame(const double n[3], double R[9]);
// The 64 canonical nodes (x' fastest) relative to the target centre.
void canonical_nodes(const double Lt[3], double nodes[kLOut][3]);
double canonical_half_width(const double Lt[3]);
// P [nodes][64]: canonical-node values -> values at the tensor grid of
// per-axis target nodes tnodes[3] (x fastest), in canonical coordinates.
void reinterp_matrix(const double Lt[3], const double R[9], const double ct[3], const std::vector<double> *tnodes,
                     std::vector<float> &P);
// Samples per history the amplitude tables allow for this geometry.
int max_samples(const LGeom &g, double cdt);

// Description of a generated history (desc rows of kLDesc doubles):
// kLGauss x (cx, cy, cz, sigma) relative to the source origin; the
// amplitude table A_g(t_j) and dA_g/dt(t_j) / (4 pi), kLGauss x kLHistT
// each; then the window centre time of sample 0 (t0, in table steps), the
// unit direction from the source centre to the target centre and the
// distance between them.
constexpr int kLDesc = 4 * kLGauss + 2 * kLGauss * kLHistT + 5;

// nh histories x samples samples: rows X [nh * samples * 4][kLIn] (fp16;
// Xf the same rows in fp32, optional) and targets Y [same][kLOut] (fp32),
// device arrays the caller allocates; desc
// (host, optional) receives the histories' descriptions.
cudaError_t learned_dataset(const LGeom &geo, uint64_t seed, int nh, int samples, double c, double dt, __half *X,
                            float *Xf, float *Y, cudaStream_t s, double *desc = nullptr);
// The linear skip: least squares (FP64 normal equations, small ridge) of Y
// on the fp32 rows Xf, into net.Wlin; Yres (optional) receives Y - Wlin x,
// the network's training targets.
cudaError_t learned_fit_linear(Mlp &net, const float *Xf, const float *Y, int rows, float *Yres, cudaStream_t s);
// Adam on minibatches drawn with replacement; cosine learning-rate decay.
cudaError_t learned_train(Mlp &net, const __half *X, const float *Y, int rows, int iterations, int batch, float lr,
                          uint64_t seed, int optin, int sms, cudaStream_t s, float *final_loss);
// rel-L2 against Y per field (rows are field-fastest) of the linear skip
// plus the network (err) and of the linear skip alone (err_lin, optional).
// With `to_nodes` the predictions at the canonical nodes are first carried
// to the label nodes the way evaluation does: y_b = Dn_b sum_a P[b][a] y_a / Ra_a
// (P [kLOut][kLOut] row b, Ra canonical-node and Dn label-node distances).
struct NodeMap {
    const float *P, *Ra, *Dn;
};
cudaError_t learned_eval(Mlp &net, const __half *X, const float *Xf, const float *Y, int rows, int optin, int sms,
                         cudaStream_t s, double err[4], double err_lin[4], const NodeMap *to_nodes = nullptr);

}  // namespace rp
