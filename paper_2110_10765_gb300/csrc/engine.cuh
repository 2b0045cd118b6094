// Batched, device-driven block Lanczos over many independent Hamiltonians
// (the batched and served forms of Fig. 1, count through eigensolve).
//
// Every problem occupies a slot.  Its CSR (FP32 values), Krylov basis Q
// [dim][MB] (FP64), work blocks and small dense state live on the device;
// the per-slot control (basis size, restart, convergence) is read and
// written by the kernels themselves, so one block-Lanczos step of every
// running slot is a fixed sequence of launches that is captured once as a
// CUDA graph and replayed.  Row work is spread over a device-resident list
// of row tiles by persistent CTAs; slots that are not running are skipped.
#pragma once

#include <memory>

#include "problem.cuh"

namespace ci {

constexpr int EB = 8;            // Lanczos block size
constexpr int ETILE = 256;       // rows per tile
constexpr int EKMAX = 16;        // eigenpairs per slot
constexpr int EMBMAX = 96;       // largest basis (Jacobi keeps T and S in shared memory)

enum SlotState { S_FREE = 0, S_INIT = 1, S_RUN = 2, S_CONV = 3, S_FAIL = 4 };
enum SlotFlag { F_CHECK = 1, F_RESTART = 2, F_FINAL = 4 };

struct Tile {
    int32_t slot;
    int32_t nr;
    int64_t r0;
};

struct SlotDev {
    int64_t dim;
    const int64_t *rp;    // [dim+1] absolute positions into col / val
    const int32_t *col;
    const float *val;
    double *Q;            // [dim][MB]
    double *W;            // [dim][EB]
    float *X, *Y;         // [dim][EB]
    int32_t k, state, flags;
    int32_t m_cur, j0, m_act, it, restarts, rank, max_iter, check_every;
    int32_t tile0, tile1;
    double hnorm, tol;
    uint64_t seed;
};

// Per-slot dense state (device arrays indexed by slot).
struct EngineDense {
    DevBuf<double> T, S, theta, Cl, Cf, Cr, G, M, R, res, evals, tres;
};

struct Engine {
    int MB = 64;                  // basis columns
    int max_slots = 0, max_tiles = 0;
    // launch shape of the persistent kernels, CTAs per SM: the tile kernels
    // (prepx, tn, QR nn, rand, restart rows, residuals) and the SpMM; picked
    // by engine_autotune.  Every tile is still handled by one CTA and every
    // row by one warp, so results do not depend on it.
    int tile_mult = 4, spmm_mult = 8;
    bool tuned = false;
    double tuned_step_ms = 0.0;   // best step time seen by the autotuner
    DevBuf<SlotDev> slots;
    DevBuf<Tile> tiles;
    DevBuf<int32_t> ntiles;       // [1]
    DevBuf<int32_t> counters;     // [4]: running slots, ...
    DevBuf<double> part;          // [max_tiles][MB*EB]
    EngineDense dn;
    std::vector<SlotDev> host_slots;
    std::vector<char> fresh;      // slots set since the last retile
    std::vector<Tile> host_tiles;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t stream = nullptr;
    int32_t *pinned_counter = nullptr;
    ~Engine();
};

void engine_create(Engine *e, int max_slots, int max_tiles, int MB, cudaStream_t s);
// Point slot i at its matrix and buffers; the slot starts in S_INIT.
void engine_set_slot(Engine *e, int i, const SlotDev &d);
void engine_free_slot(Engine *e, int i);
// Rebuild the tile list from the slots that are not free.
void engine_retile(Engine *e);
// Initialise the start blocks of every S_INIT slot (random, orthonormal).
void engine_init_slots(Engine *e);
// Pick the launch shape by timing real steps of the running slots with each
// candidate (two steps per candidate: capture, then a timed replay); the
// choice is cached per device and workload size.  Returns the steps taken.
int engine_autotune(Engine *e);
// One block-Lanczos step of every running slot (graph replay).
void engine_step(Engine *e);
// Number of running slots (synchronises the engine stream).
int engine_running(Engine *e);
// Copy slot results (evals, estimates) to the host and compute the FP64
// residuals ||H x - theta x|| of finished slots.
void engine_results(Engine *e, int i, double *evals, double *res_est, double *res_true, int *iters, int *state);
void engine_true_residuals(Engine *e);

}  // namespace ci
