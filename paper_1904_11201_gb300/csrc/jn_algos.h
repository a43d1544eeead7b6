// Internal entry points of the join algorithms (device-resident columns).
#pragma once

#include <memory>
#include <vector>

#include "jn_common.cuh"

namespace jnx {

enum RunMode { MODE_COUNT = 0, MODE_AGG = 1, MODE_EMIT = 2 };

// One table with every column already in device memory.
template <typename K>
struct Cols {
    const K* key;
    const K* key2;
    const int32_t* pay;  // NULL = row index
    int64_t n;
    bool host = false;   // columns read in place from page-locked host memory
};

// Where the pairs of an emitting run go (see jn.h's output convention).
struct OutPlan {
    jn_pair** user_out = nullptr;
    uint64_t capacity = 0;
    uint64_t* n_out = nullptr;
    jn_pair* dev = nullptr;      // device buffer the kernels write
    bool host_copy = false;      // caller buffer is host memory, filled by a copy
    bool lib_alloc = false;      // library allocated the result
    bool mapped = false;         // caller buffer is page-locked host memory written in place
    bool copied = false;         // the run already copied the pairs to the caller's host buffer
};

// Sizes the output for `m` pairs (allocating or checking the caller buffer).
jn_status out_prepare(jn_ctx* c, Scratch& s, uint64_t m, OutPlan& plan);
// Copies to a host buffer when needed and publishes the result.
jn_status out_finish(jn_ctx* c, uint64_t m, OutPlan& plan);

struct RunResult {
    uint64_t count = 0;
    uint64_t checksum = 0;
};

// R rows one hash-join work item holds in shared memory, by key type.
int hash_cap(int32_t key_type);

template <typename K>
jn_status run_hash(jn_ctx* c, const Cols<K>& R, const Cols<K>& S, int mode, OutPlan* plan,
                   RunResult* res, bool sort_merge = false);

// A batch of joins run as one: prepare() (all passes up to the exact
// counts) fills total and the per-join offsets; emit() writes the pairs to
// out[0 .. total).  The object owns the batch's scratch between the two.
struct BatchRun {
    uint64_t total = 0;
    std::vector<uint64_t> offsets;  // joins + 1 offsets inside this run's pairs
    virtual ~BatchRun() {}
    virtual jn_status emit(jn_ctx* c, jn_pair* out) = 0;
};

template <typename K>
jn_status batch_hash_prepare(jn_ctx* c, int n, const Cols<K>* Rs, const Cols<K>* Ss, std::unique_ptr<BatchRun>* run);

template <typename K>
jn_status batch_band_prepare(jn_ctx* c, int m, const Cols<K>* Rs, const Cols<K>* Ss, const int* ops,
                             const int64_t* bands, std::unique_ptr<BatchRun>* run);

// Captures a sequence of launches on the context's private stream and replays
// it as a CUDA graph on the context's stream (or runs it directly when graphs
// are off).  The caller's stream may be the legacy default stream, which
// cannot itself be captured.
struct GraphPhase {
    jn_ctx* c;
    bool on;
    cudaStream_t user = nullptr;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t x = nullptr;
    GraphPhase(jn_ctx* ctx, bool graphs) : c(ctx), on(graphs) {}
    ~GraphPhase();
    jn_status begin();
    jn_status end_and_run();
    void abort();
};

template <typename K>
jn_status run_nlj(jn_ctx* c, const Cols<K>& R, const Cols<K>& S, const jn_pred& pred, int mode,
                  OutPlan* plan, RunResult* res);

template <typename K>
jn_status run_theta(jn_ctx* c, const Cols<K>& R, const Cols<K>& S, int op, int64_t band, int mode,
                    OutPlan* plan, RunResult* res);

}  // namespace jnx
