// Plan state shared by the host-side translation units of the library.
#pragma once
#include <cuda_runtime.h>

#include <functional>
#include <string>
#include <vector>

#include "../../include/polyspec.h"
#include "kernels.h"

struct CcTiles {
    std::vector<PsTile> tiles;
    std::vector<int> field_ids;
    std::vector<short4> rowf, colf;  // up to three factors each (-1: none)
    std::vector<int64_t> slot;  // per bin: tile * 64 * 64 + r * 64 + c
};

// Largest number of shells a plan takes.  Host tables pack shell and field-slot
// numbers into fixed-width keys that rely on it (checked where they are packed).
constexpr int kPsMaxShells = 128;

struct TcState;     // tensor-core contraction state (contract_tc.cu)
struct AdjTables;  // adjoint entry tables (adjoint.cu)

struct poly_plan_s {
    // configuration
    int N = 0;
    double L = 0;
    int order = 0;
    int nshell = 0;
    std::vector<double> edges;
    poly_precision prec = POLY_FP32;
    unsigned flags = 0;
    int is_double = 0;
    int K = 0;  // largest integer wavevector component inside the outer shell
    int ell = 0;     // multipole of the first leg (0: the monopole estimator)
    int nfield = 0;  // field slots in the cell-tiled array: nshell, or 2 nshell with the weighted set for ell > 0
    int device = -1;
    int sms = 0;
    // bins and counts (host)
    int64_t nbins = 0;
    std::vector<int32_t> bins;
    std::vector<int64_t> counts;
    // device tables
    void* d_tw_fwd = nullptr;  // Cx<double>[N], e^{-2 pi i m/N}
    void* d_tw_inv = nullptr;  // Cx<double>[N], e^{+2 pi i m/N}
    void* d_lines = nullptr;   // short4 per (shell, line): ky, kz, a, b
    int* d_line_off = nullptr; // nshell + 2 offsets (last slot: union of all shells)
    std::vector<int> line_off; // host copy
    std::vector<int> shell_kz; // largest kz of each shell's lines (host)
    int* d_shell_kz = nullptr; // the same on the device
    int max_lines = 0;         // largest line count of one shell (or of the union)
    void* d_xpre = nullptr;    // x-pass output of the inverse transform
    size_t xpre_lines = 0;     // lines the x-pass buffer holds (indexed by global line offset)
    // CUDA-core contraction
    CcTiles cc;
    void *d_cc_tiles = nullptr, *d_cc_field_ids = nullptr, *d_cc_rowf = nullptr, *d_cc_colf = nullptr,
         *d_cc_slot = nullptr;
    int cc_nsplit = 1;
    int64_t cc_cps = 0, cc_slot_stride = 0;
    // workspace
    void* d_W = nullptr;       // forward intermediate, N x (2K+1)(K+1) complex
    void* d_fhat = nullptr;    // pruned half spectrum, (2K+1)(K+1)(2K+1) complex
    void* d_fhat_w = nullptr;  // the same weighted by L_ell(kz/|q|) (ell > 0)
    void* d_fields = nullptr;  // nshell x N^3 real
    void* d_spill = nullptr;   // plane-kernel overflow (FP64 at large K)
    double* d_partial = nullptr;
    double* d_S = nullptr;
    int64_t* d_counts = nullptr;
    void* d_in_stage = nullptr;    // host-buffer entry point staging
    double* d_out_stage = nullptr;
    // adjoint workspace (allocated on first backward)
    void* d_G = nullptr;      // nshell x N^3 real
    void* d_ghat = nullptr;   // union spectrum
    AdjTables* adj = nullptr;
    // disconnected part of the trispectrum (allocated on first use)
    int32_t* d_bins = nullptr;     // nbins x order, 1-based shells
    double* d_shell_power = nullptr;
    // full-shape trispectrum scratch (mode lists, diagonal table, accumulators; grown on demand)
    void* d_tf = nullptr;
    size_t tf_bytes = 0;
    // tensor-core contraction: state, and its tunable shape (poly_plan_tune)
    TcState* tc = nullptr;
    int tc_max_mt = 4;    // largest number of M tiles per CTA group
    int tc_cta_mult = 4;  // CTA budget = SM count x tc_cta_mult / 2 (two waves balance the tail best)
    // instrumentation
    int64_t launches = 0;
    bool timing = false;
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    bool ev_recorded = false;
    // every device allocation owned by the plan
    std::vector<void*> allocations;
    std::vector<size_t> allocation_bytes;  // size of each entry of allocations
};
typedef poly_plan_s PsPlan;

poly_status ps_alloc(PsPlan* p, void** ptr, size_t bytes);
void ps_free(PsPlan* p, void* ptr);  // frees one allocation made by ps_alloc (NULL: no-op)
void ps_set_last_error(const std::string& msg);
// host-side tables (plan.cpp)
void enumerate_bins(int nshell, const std::vector<double>& edges, int order, bool all_sorted, std::vector<int32_t>& out);
void build_lines(const PsPlan* p, const double* e, int s, std::vector<short>& lines);
void build_cc_tiles(PsPlan* p, CcTiles& t, int first_shift = 0);
// the adjoint's entry tables (adjoint.cu); host only
void ps_adj_entries(const PsPlan* p, std::vector<int>& moff, std::vector<short4>& ent, std::vector<int>& eoff,
                    std::vector<int>& ebins);
// host part of plan creation (checks, bins, shell line tables, contraction tiles); no device call
poly_status ps_plan_host_tables(PsPlan* p, int N, double L, int order, int nshell, const double* edges,
                               poly_precision prec, unsigned flags, int ell, std::vector<short>& lines);
poly_status ps_fields(PsPlan* p, const void* delta, cudaStream_t st);
// true when the x-pass buffer holds shells [s0, s0 + ns) (global line offsets)
bool ps_xpre_fits(const PsPlan* p, int s0, int ns);
poly_status ps_sums(PsPlan* p, bool absval, cudaStream_t st);
poly_status ps_estimate_impl(PsPlan* p, const void* delta, double* out, double* scale, cudaStream_t st);
double ps_norm(const PsPlan* p);

// contract_tc.cu
poly_status ps_tc_prepare(PsPlan* p);
poly_status ps_tc_sums(PsPlan* p, cudaStream_t st);
void ps_tc_free(PsPlan* p);
double ps_tc_executed_flops(const PsPlan* p);
poly_status ps_check_device_error(PsPlan* p);

// adjoint.cu
void ps_adj_free(PsPlan* p);
int ps_adj_device_error(PsPlan* p);  // nonzero: the tensor-core adjoint kernel timed out
// trispectrum_full.cu
poly_status ps_trispectrum_full_impl(PsPlan* p, const void* delta, const int32_t* k, int nd, const double* dedges,
                                     double* T_out, int64_t* counts_out, double* scale_out, cudaStream_t st);
poly_status ps_backward_impl(PsPlan* p, const void* delta, const double* dL_dB, void* dL_ddelta, cudaStream_t st);
// batched.cpp
poly_status ps_batched_impl(const poly_plan* plans, const void* const* fields, double* const* outs, int count,
                            cudaStream_t st);
void ps_batched_forget(const PsPlan* p);  // drop cached graphs that use p
