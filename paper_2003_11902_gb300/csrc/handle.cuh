// The single-colony handle behind the C ABI, shared by the runtime and the
// batched-colony front end.
#pragma once

#include <string>

#include "internal.cuh"
#include "mmas.h"
#include "twoopt.cuh"

struct mmas_handle {
    int device = 0;
    int n = 0, m = 0, cl = 0, ld = 0;
    mmas_params p{};
    double p_root = 0.0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int num_sms = 0;
    size_t smem_optin = 0;

    int2 *xy = nullptr;
    int32_t *dist = nullptr;
    float *eb = nullptr, *tau = nullptr, *wmat = nullptr, *cwinv = nullptr;
    int32_t *cand32 = nullptr;
    uint16_t *cand16 = nullptr;
    int32_t *tours = nullptr, *lens = nullptr, *gb_tour = nullptr, *nn_tour = nullptr;
    int2 *nbr = nullptr;
    mmas::Scalars *sc = nullptr;
    int *maxd = nullptr;
    int32_t maxd_val = 0;            // the instance's largest distance
    float *ebt = nullptr;            // [maxd_val + 1] eta^beta of each distance value, or null
    int32_t *ext_tour = nullptr, *ext_len = nullptr;
    uint32_t *ext_bad = nullptr;     // set when a device-side tour was refused (skip that update)
    int32_t *nnd = nullptr;
    int32_t xe = 0;                  // reach-list length of the greedy fallback (0: none)
    int32_t *xl32 = nullptr;         // [n][xe]
    uint2 *xlw = nullptr;            // [n][xe]
    float *xlb = nullptr;            // [n]
    uint2 *xxw = nullptr;            // [n][REACH_EXTRA]
    int32_t *xxn = nullptr;          // [n]
    int32_t *xhot = nullptr;         // [n]
    int32_t fe = 0, fp = 0;          // far list of the greedy fallback: entries past the reach list, row pitch
    uint16_t *xf16 = nullptr;        // [n][fp]
    float *xfb = nullptr;            // [n]
    mmas::FarList *far = nullptr;    // device copy of {xf16, xfb, fp} for the construction
    mmas::Scalars *h_sc = nullptr;  // pinned mirror of *sc
    int32_t *h_tour = nullptr;      // pinned staging of the best tour

    mmas::ConstructArgs cargs{};
    mmas::ConstructPlan cplan{};
    mmas::BestArgs bargs{};
    mmas::ScoreArgs sargs{};
    mmas::TwoOptArgs targs{};
    mmas::UpdateArgs uargs{};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    bool timing = false;
    bool timed_run = false;
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    std::string err;
};

namespace mmas {
// Host-side checks of one colony's instance and parameters (no device work);
// on failure the message is the calling thread's mmas_last_error(NULL).
mmas_status validate_colony(const mmas_instance *inst, const mmas_params *params);
}  // namespace mmas
