/*
 * cur_batch.h -- batched IterativeCUR: many independent decompositions
 * (Algorithm 1 of arXiv 2509.21963, residuals through Lemma 1, Sec. 4.2) in
 * one persistent cooperative kernel.
 *
 * The paper treats one matrix at a time; it has no batched form.  The method
 * per job is exactly that of cur_run (cur.h): same Gaussian sketch for the
 * same seed (see cur_step_gaussian in cur_steps.h), same LUPP selection rules,
 * same stopping test rho = ||S^col||_F / ||G A||_F <= eps (Sec. 3.3), the core
 * U = A(I,J)^+ by Householder QR with column pivoting at exit (Sec. 3.3).
 * Only the schedule differs: the GPU is cut into teams of co-resident CTAs,
 * each team takes jobs from a device-side queue (largest estimated work
 * first) and runs every step of a job, synchronising through bounded
 * device-side barriers, so a whole batch is one launch (replayed from a
 * captured CUDA graph when the runtime allows it).
 *
 * Conventions are those of cur.h: row-major matrices, 0-based int64 indices,
 * every call returns a cur_status and leaves a one-line text in
 * cur_last_error(ctx).  A batch belongs to the context it was created on and
 * is not thread-safe.
 */
#ifndef CUR_BATCH_H
#define CUR_BATCH_H

#include <stddef.h>
#include <stdint.h>

#include "cur.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cur_batch cur_batch;

/* One decomposition request.
 *   A            device, m x n, row stride lda >= n, of the batch's dtype;
 *                borrowed: read only, valid and unchanged until the batch is
 *                freed (every cur_batch_run reads it again).
 *   m, n         >= 1.
 *   tol          eps > 0 (NaN or <= 0: CUR_EINVAL); eps >= 1 gives rank 0.
 *   block_size   1 <= b <= 64.
 *   sketch_size  c with b <= c <= 128; 0 selects floor(1.1 b) (Sec. 1.1).
 *   seed         key of the Gaussian sketch.
 *   max_rank     cap on |I| = |J| (<= 0: min(m, n)). */
typedef struct cur_batch_job {
  const void *A;
  int64_t m, n, lda;
  double tol;
  int32_t block_size;
  int32_t sketch_size;
  uint64_t seed;
  int64_t max_rank;
} cur_batch_job;

/* Validate the jobs (host array of njobs >= 1 entries, copied), size the
 * outputs and scratch, and choose a default schedule (team size from the
 * largest job).  dtype: CUR_F64 or CUR_F32 for every A of the batch.
 * Device memory: outputs sum_j (2 r_j + r_j^2 + r_j / b_j) words with
 * r_j = min(m_j, n_j) (or max_rank), plus scratch per team sized by the
 * largest job; CUR_EBUDGET if that exceeds the context's budget.
 * Errors: CUR_EINVAL names the first offending job. */
int cur_batch_create(cur_ctx *ctx, const cur_batch_job *jobs, int64_t njobs, int dtype,
                     cur_batch **out);

/* Release the batch and its device memory.  NULL is a no-op. */
void cur_batch_free(cur_batch *batch);

/* Schedule: `team` co-resident CTAs of 256 threads per job (1..32; 0 keeps
 * the current value).  Reallocates the team scratch; invalidates the graph. */
int cur_batch_set_team(cur_batch *batch, int team);

/* Schedule with two team classes: nbig teams of team_big CTAs take the
 * big_cut largest jobs (by estimated work; the queue is ordered largest
 * first), then help with the rest; the remaining co-resident CTAs form teams
 * of `team` CTAs that take only the other jobs.  So a job's team size follows
 * its size class.  nbig = 0 is cur_batch_set_team(batch, team).  CUR_EINVAL
 * when the big teams leave no room for one team of `team` CTAs.  Reallocates
 * the team scratch; invalidates the graph. */
int cur_batch_set_classes(cur_batch *batch, int team, int team_big, int nbig, int64_t big_cut);

/* The big-team class of the current schedule (team_big = nbig = big_cut = 0
 * when there is one class). */
int cur_batch_get_classes(const cur_batch *batch, int *team_big, int *nbig, int64_t *big_cut);

/* Tile of the residual products inside the batch kernel (the Lemma 1
 * products S^row = A(:,J_k) - L Rt(:,J_k) and the factor/sketch updates of
 * Sec. 4.2): each thread forms tile_n (4 or 8) outputs per pass over the
 * staged inner dimension.  The same arithmetic either way (each output is one
 * FP64 dot product in the same order); only registers and shared-memory
 * reuse differ.  Invalidates the graph.  CUR_EINVAL for other values. */
int cur_batch_set_tile(cur_batch *batch, int tile_n);
int cur_batch_get_tile(const cur_batch *batch, int *tile_n);

/* Current schedule: team size, CTAs launched, teams, whether launches replay a
 * captured graph (1) or are direct cooperative launches (0). */
int cur_batch_get_schedule(const cur_batch *batch, int *team, int *grid, int *teams,
                           int *graph);

/* Autotuner: for each candidate team size (candidates: host array of ncand
 * sizes, or NULL for {1, 2, 4, 8, 16}) capture the launch graph first, then
 * run the whole batch twice, timing each run with CUDA events; the faster run
 * is the candidate's time.  After the single-class candidates it tries, on
 * top of the fastest of them, two-class schedules (cur_batch_set_classes):
 * 1 or 2 big teams of 8 or 16 CTAs (larger than the small teams) serving the
 * largest jobs up to the big teams' share of the CTAs in estimated work,
 * then the other product tile (cur_batch_set_tile) on the fastest schedule.
 * The fastest schedule is kept; *best_team receives its small-team size.  Every trial is
 * a complete, valid run, so the results of the last trial are available
 * afterwards.  *best_team and *best_ms (optional) receive the choice and its
 * time. */
int cur_batch_tune(cur_batch *batch, const int *candidates, int ncand, int *best_team,
                   double *best_ms);

/* Enqueue one run of the whole batch on the context's stream (ordered after
 * the work already on it) and return without waiting. */
int cur_batch_launch(cur_batch *batch);

/* Wait for the last launch, read the per-job records back and translate a
 * device-side failure (CUR_ETIMEOUT if a team barrier ran out of its budget).
 * Returns CUR_OK when the launch completed, whatever the jobs' own statuses. */
int cur_batch_wait(cur_batch *batch);

/* cur_batch_launch followed by cur_batch_wait. */
int cur_batch_run(cur_batch *batch);

/* SM cycles the team leaders spent per phase in the last completed run,
 * summed over teams: [0] sketch (G and G A), [1] column selection, [2] row
 * residual, [3] row selection and N^+, [4] factor and sketch updates, [5] core
 * factorisation, [6] core solve, [7] number of jobs.  cycles: host array of
 * nphase (<= 8) entries. */
int cur_batch_phase_cycles(const cur_batch *batch, double *cycles, int nphase);

/* SM cycles the job took in the last completed run (its team leader's clock,
 * from taking the job to finishing it). */
int cur_batch_job_cycles(const cur_batch *batch, int64_t job, int64_t *cycles);

/* Per-job results of the last completed run (job in [0, njobs)).
 * status: CUR_OK, CUR_TOL_UNREACHED (stopped at max_rank), CUR_ENONFINITE
 * (G A not finite), CUR_ETIMEOUT or CUR_ECUDA (internal failure). */
int cur_batch_job_result(const cur_batch *batch, int64_t job, int64_t *rank, int64_t *iters,
                         double *rho, int *status);

/* Device arrays of a job, valid until the next run or cur_batch_free:
 * I and J (rank entries, selection order), U (rank x rank row-major FP64,
 * |J| x |I|, so that A ~ A(:,J) U A(I,:)), rho after each iteration. */
const int64_t *cur_batch_I(const cur_batch *batch, int64_t job);
const int64_t *cur_batch_J(const cur_batch *batch, int64_t job);
const double *cur_batch_U(const cur_batch *batch, int64_t job);
const double *cur_batch_rho_history(const cur_batch *batch, int64_t job);

/* Copy a job's I, J (rank entries each), U (rank^2) and rho history
 * (iterations entries) into host buffers (any may be NULL).  Synchronous. */
int cur_batch_copy_job(const cur_batch *batch, int64_t job, int64_t *I, int64_t *J, double *U,
                       double *rho_history);

#ifdef __cplusplus
}
#endif

#endif /* CUR_BATCH_H */
