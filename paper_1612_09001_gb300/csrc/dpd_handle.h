// The handle behind dpd_handle (include/dpd.h), shared by the libdpd API
// translation units.  Not part of the public C ABI.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

#include "dpd_internal.h"

// Device workspace of dpd_estimate, grown on demand.
struct EstimateWorkspace {
    int cpp = 0;                  // Gram CTAs per problem the partials were sized for
    int nprob = 0;                // problems the per-problem arrays were sized for
    int64_t nsamp = 0;            // samples the y / e buffers hold
    void *probs = nullptr;        // GramProblem[nprob]
    float *partials = nullptr;    // [nprob * cpp][kGramRows][kGramPartCols]
    double *S = nullptr;          // [nprob][kGramS][kGramPartCols]: summed P and Q blocks
    double *Clag = nullptr;       // [nprob][kLagEntries]: summed lag sums (tensor-core Gram)
    double2 *G = nullptr, *g = nullptr, *L = nullptr, *h64 = nullptr, *delta = nullptr;
    double *d = nullptr, *tt = nullptr;
    int *info = nullptr;
    float2 *hf = nullptr;         // coefficients of the refinement pass (complex64)
    float *tab = nullptr;         // their forward table
    float2 *y = nullptr, *e = nullptr;
    double *norm_part = nullptr;  // 2 * kFwdNormSlots partial sums, 2 results, a counter
    // orthogonal-polynomial basis (DPD_BASIS_ORTHOGONAL)
    float *ubasis = nullptr;      // [nprob][kUSize] basis coefficients used by the Gram kernels
    double *ubasis64 = nullptr;   // the same values in FP64, for the coefficient transforms
    double *mom = nullptr;        // [nprob][kMomK] power sums of |u|^2
    double *mom_part = nullptr;   // [nprob][kMomBlocks][kMomK]
    double2 *hm64 = nullptr;      // [nprob][K] monomial-basis coefficients / transformed right-hand sides
    // single problem: explicit inverse of the Cholesky factor for the solves
    double2 *Linv = nullptr;      // K x K
    double2 *tmpv = nullptr;      // K
    bool use_inverse = false;     // refinement solves through Linv (problem 0 only)
    // pinned host copies read back by dpd_estimate (single problem)
    int hK = 0;                   // K the host buffers were sized for
    double2 *h_G = nullptr;       // Gram matrix G, K x K (condition estimate on the host)
    double2 *h_Linv = nullptr;    // inverse Cholesky factor of D G D, K x K
    int *h_info = nullptr;        // pivot status of the factorisation
    double *h_norm = nullptr;     // ||t - Psi h||^2, ||t||^2
    cudaEvent_t ev_G = nullptr;   // h_G has landed
    // batched refinement (dpd_estimate_batched): per-problem forward tables,
    // work lists of the batched forward and coefficient-gradient launches
    float *tabb = nullptr;        // [problems][tstride]
    size_t tabb_cap = 0;
    void *bstreams = nullptr;     // dpd::BatchStream [problems]
    void *bitems = nullptr;       // dpd::BatchItem [items]
    void *badj = nullptr;         // dpd::AdjArgs [problems]
    float2 *bpart = nullptr;      // coefficient-gradient partials, [problems][K]
    size_t bprob_cap = 0, bitems_cap = 0;
    cudaEvent_t ev_L = nullptr;   // h_info (and h_Linv) have landed
};

// Device staging of dpd_apply_host's copy / compute pipeline, created on first use.
constexpr int kHostSlots = 3;
struct HostPipeline {
    int64_t chunk = 0;                         // samples per chunk (capacity excludes the history)
    float2 *in[kHostSlots] = {};
    float2 *out[kHostSlots] = {};
    cudaStream_t streams[kHostSlots] = {};
    cudaEvent_t done[kHostSlots] = {};
    cudaEvent_t start = nullptr;
};

struct dpd_filter {
    int P, Q, M;
    int Bp, Bq, B, T, K;
    int device;
    int sm_count;
    float2 *d_h;      // K complex coefficients, stacking order of Sec. 2.2
    float *d_tab;     // widely-linear table for the forward kernels
    int *d_status;    // kernel error word
    float2 *d_hist;   // streaming history: the kHalo input samples before the next dpd_apply_stream
    double *d_loss_part;   // dpd_sq_error: per-block FP64 partial sums (kLossBlocks)
    float *d_adj_tab; // adjoint (derivative-polynomial) table
    float2 *d_partials;  // coefficient-gradient workspace: rows_max x K complex
    int rows_max;
    bool has_coeffs;
    bool host_tab_valid;  // h_tab / h_adj_tab mirror d_tab / d_adj_tab
    bool tab_from_device = false;   // ... copied back after a device-side dpd_set_coeffs
    bool tab_pending = false;       // a copy back is queued (ev_tab marks its end)
    dpd::HostTab h_tab;
    float h_adj_tab[dpd::kMaxAdjTabFloats];
    float *h_tab_pin = nullptr;     // pinned landing buffers of the copy back
    float *h_adj_pin = nullptr;
    cudaEvent_t ev_tab = nullptr;
    dpd::FwdLaunch fwd;
    bool fwd_auto = true;
    int est_basis = 0;      // DPD_BASIS_MONOMIAL or DPD_BASIS_ORTHOGONAL (least-squares estimates)   // default launch shape: shrink the tile for short inputs (off once set explicitly)
    dpd::AdjLaunch adj;
    EstimateWorkspace est;
    HostPipeline host;
};

void free_estimate_workspace(EstimateWorkspace &w);
void free_host_pipeline(HostPipeline &p);


namespace dpd {
constexpr int kLossBlocks = 296;   // 2 per SM at 148-152 SMs
// loss[0] = (float)(scale * sum |y - g x|^2) (FP64 sum, fixed order); gy = 2 scale (y - g x) if non-null.
cudaError_t launch_sq_error(const float2 *y, const float2 *x, int64_t n, float2 g, double scale, double *part,
                            float *loss, float2 *gy, cudaStream_t s);
// Streaming head: recompute y[0 .. min(T-1, n)) with the kHalo samples in hist
// as the history before x[0] (the forward kernels assume zero history), then
// hist <- the last kHalo samples of (hist ++ x).  One warp; runs after the
// forward launch on the same stream.
cudaError_t launch_stream_head(const float *tab, int B, int T, const float2 *x, int64_t n, float2 *hist,
                               float2 *y, cudaStream_t s);
}  // namespace dpd
