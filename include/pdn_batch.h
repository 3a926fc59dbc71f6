/* Batched explicit PDN impact steps: many independent plates, each with its
 * own mesh, material, stable step and striker, advanced together by one
 * persistent kernel per launch (a work queue of tiles over all plates).
 *
 * The method is the one of pdn.h (Algorithm 1 per step, per plate); a batch
 * only changes how the work is scheduled on the GPU.  The paper runs its
 * impact cases one after another on a cluster (Sec. 3); here every pass
 * walks four phases over the tiles of all plates:
 *   1. contact detection and projection of every plate's surface nodes;
 *   2. hex8 and interface internal forces (all plates' element tiles);
 *   3. CSR gather and node update (all plates' node tiles);
 *   4. the tail of every plate: its own reaction sum (a segmented reduction:
 *      one block per plate), commit / repeat (Algorithm 2) / halt, and its
 *      striker update with its own time step;
 * Two schedules: a grid-wide barrier between phases, or dataflow (one queue
 * of pass/phase/tile positions; a tile waits only until the previous phase of
 * its own plate is complete, so one plate's gather overlaps another plate's
 * elements).  Every wait is bounded in time.  The launch is cooperative (all
 * blocks resident), captured in a CUDA graph, and repeats passes until every
 * plate has reached its target step.  Each plate follows the same device
 * state machine and the same per-item source code as pdn_step, with the
 * same fixed reduction orders, so a plate stepped in a batch follows the
 * plate stepped alone to floating-point rounding (the compiler may contract
 * multiply-adds differently in different kernel instantiations) and
 * repeated runs of one schedule are bitwise identical.
 *
 * The schedule, tile size, blocks per SM and the kernel's register budget are
 * chosen by an autotuner on the first pdn_batch_step (timing internal-force
 * passes, which leave the state unchanged); the environment variable
 * PDN_BATCH_SCHEDULE="s" or "s,r" restricts it to schedule s (0 barrier, 1
 * dataflow) and register variant r (see pdn_batch_info.reg_variant). */
#ifndef PDN_BATCH_H
#define PDN_BATCH_H

#include <stdint.h>

#include "pdn.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pdn_batch pdn_batch;

/* Schedule and counters of a batch. */
typedef struct {
  int32_t n_plates;
  int32_t precision;
  int32_t status;          /* sticky: PDN_OK or the first error (see pdn_batch_step) */
  int32_t tuned;           /* 1 once the autotuner has chosen the schedule */
  int32_t blocks_per_sm;   /* persistent blocks per SM of the chosen schedule */
  int32_t tile_items;      /* items (nodes or elements) per tile */
  int32_t reg_variant;     /* register budget: 0 = 128/thread (4 blocks/SM), 1 = 255 */
  int32_t grid;            /* blocks of the persistent launch */
  int32_t graph;           /* 1: launches replay a captured CUDA graph */
  int32_t n_candidates;    /* schedules timed by the autotuner */
  int64_t n_tiles[4];      /* tiles of the contact, element, gather and tail phases */
  int64_t launches;        /* persistent launches so far */
  int64_t passes;          /* passes executed so far (all launches) */
  double tune_ms[16];      /* internal-force pass time of each candidate (ms) */
  int32_t tune_bps[16];    /* candidate: blocks per SM */
  int32_t tune_tile[16];   /* candidate: items per tile */
  int32_t tune_var[16];    /* candidate: register variant */
  int32_t dataflow;        /* chosen schedule: 0 grid barriers between phases, 1 dataflow
                              (per-plate phase dependencies, no barrier) */
  int32_t pad;
  int32_t tune_flow[16];   /* candidate: schedule */
} pdn_batch_info;

/* Create a batch of n_plates (1..4096) plates on the current device.
 * meshes[p] and mats[p] describe plate p exactly as for pdn_init_mesh; the
 * options (precision, laws, time-step rule, stream, ...) are common to all
 * plates, and dt = 0 selects each plate's own stable step.  All device
 * memory of the plates is allocated here.  On failure *out is NULL and
 * pdn_batch_last_error(NULL) says why. */
int pdn_batch_init(pdn_batch **out, int32_t n_plates, const pdn_mesh_desc *meshes,
                   const pdn_material *mats, const pdn_options *opt);

/* Context of plate p, owned by the batch (NULL if p is out of range).  Use
 * it with pdn_set_impactor, pdn_contact_force, pdn_damage_field,
 * pdn_get_state, pdn_set_state, pdn_get_contact, pdn_internal_force and
 * pdn_get_info.  pdn_step on it advances that plate alone; never pass it
 * to pdn_destroy. */
pdn_ctx *pdn_batch_plate(pdn_batch *b, int32_t p);

/* Advance every plate by nsteps of its own time step (Algorithm 1 per plate,
 * step repetitions for released contact nodes as in pdn_step).  Every plate
 * needs a striker (PDN_E_STATE otherwise).  Returns after the work has
 * completed.  Errors: PDN_E_NONFINITE or PDN_E_RELEASE_LIMIT of any plate
 * (that plate halts; the message names it; the others keep their progress),
 * PDN_E_TIMEOUT when a grid barrier wait gave up (the batch is then unusable:
 * sticky), PDN_E_CUDA. */
int pdn_batch_step(pdn_batch *b, int64_t nsteps);

/* Schedule and counters; see pdn_batch_info. */
int pdn_batch_get_info(pdn_batch *b, pdn_batch_info *info);

/* Testing the bounded barrier: one persistent launch in which block 0 never
 * arrives at the first barrier, with every plate idle, so that the other
 * blocks give up after timeout_ms milliseconds.  Returns PDN_E_TIMEOUT when
 * the wait ran out as designed (the batch stays usable: nothing was
 * computed), PDN_OK if it did not, or another error. */
int pdn_batch_test_barrier_timeout(pdn_batch *b, double timeout_ms);

/* Release the batch and every plate context.  NULL is ignored. */
void pdn_batch_destroy(pdn_batch *b);

/* Message of the last error of b, or of the last failed pdn_batch_init in
 * this thread when b is NULL. */
const char *pdn_batch_last_error(const pdn_batch *b);

#ifdef __cplusplus
}
#endif

#endif /* PDN_BATCH_H */
