/*
 * messi_oracle.h -- plain FP64 CPU reference of the MESSI exact k-NN method.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or
 * call this code: only tests/, __graft_entry__.smoke() and bench.py's CPU
 * baseline leg use it.  It shares no code, header, table or constant with the
 * CUDA library in paper_2110_07519_gb300/.
 *
 * Every routine is the plain definition the paper gives (section cited beside
 * each declaration), written for obviousness, not speed:
 *   - FP64 throughout, no FMA contraction (built with -ffp-contract=off),
 *   - sequential sums in index order,
 *   - no blocking, fusion or reordering beyond what the definition states.
 *
 * Conventions: a series is n contiguous float32 values; w segments of
 * m = n / w points; cardinality c = 2^b symbols; symbol 0 is the lowest
 * y-region.  Breakpoint table beta[0..c-2] holds beta_1..beta_{c-1}.
 */
#ifndef MESSI_ORACLE_H
#define MESSI_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* iSAX breakpoints (Sec. 2.2, "iSAX Representation": the y-axis is split
 * into c equiprobable regions of N(0,1)).  beta[j-1] = the double nearest
 * PhiInv(j / c) for j = 1..c-1, found by bisection on doubles with Phi
 * evaluated in double-double arithmetic from its Maclaurin series. */
void orc_breakpoints(int card, double *beta);

/* PAA (Sec. 2.2): paa[s] = mean of x[s*m .. s*m+m-1], FP64 sequential sum,
 * divided by m. */
void orc_paa(const float *x, int n, int w, double *paa);

/* SAX symbol (Sec. 2.2): sym[s] = #{ j in 1..c-1 : beta_j <= paa[s] }.
 * A value equal to a breakpoint goes to the upper region. */
void orc_sax(const double *paa, int w, int card, const double *beta, uint8_t *sym);

/* Summarise many rows: PAA then SAX for each of N rows of length n. */
void orc_summarize(const float *data, int64_t N, int n, int w, int card,
                   const double *beta, uint8_t *sax /* N*w */);

/* Interleaved iSAX key (Sec. 2.2 "ParIS+ Index": a node refines one segment
 * by one more bit at a time).  Bit position p (0 = most significant of 128)
 * with p = j*w + s holds bit (b-1-j) of sym[s]; key[0] holds bits 0..31. */
void orc_isax_key(const uint8_t *sym, int w, int card, uint32_t key[4]);

/* Squared Euclidean distance (Sec. 2.1): sum_t (q_t - x_t)^2 in FP64,
 * sequential over t. */
double orc_ed2(const float *q, const float *x, int n);

/* ED lower bound from the query PAA and a candidate's iSAX word
 * (Property 1, Sec. 4): m * sum_s d_s^2 with d_s the distance from paa_q[s]
 * to the candidate's region [beta_sym, beta_{sym+1}] (0 inside).  Squared. */
double orc_mindist_ed2(const double *paa_q, const uint8_t *sym, int w, int m,
                       int card, const double *beta);

/* LB_Keogh envelope (Sec. 3.4): U_i = max q_j, L_i = min q_j over
 * j in [i-r, i+r] clipped to [0, n-1]. */
void orc_envelope(const float *q, int n, int r, double *U, double *L);

/* LB_Keogh (Sec. 3.4), squared: sum_i (c_i-U_i)^2 if c_i > U_i,
 * (c_i-L_i)^2 if c_i < L_i, else 0. */
double orc_lb_keogh2(const double *U, const double *L, const float *x, int n);

/* DTW lower bound from the envelope PAA and an iSAX word (Sec. 3.4, the
 * ABOVE / BELOW / IN cases): per segment, ABOVE gives beta_sym - paaU[s]
 * when paaU[s] < beta_sym, BELOW gives paaL[s] - beta_{sym+1} when
 * paaL[s] > beta_{sym+1}, IN gives 0; result m * sum d_s^2 (squared). */
double orc_mindist_dtw2(const double *paaU, const double *paaL, const uint8_t *sym,
                        int w, int m, int card, const double *beta);

/* DTW under a Sakoe-Chiba window r (Sec. 3.4), squared cost:
 * D(i,j) = (q_i - x_j)^2 + min(D(i-1,j), D(i,j-1), D(i-1,j-1)) for
 * |i-j| <= r, +inf outside; result D(n-1, n-1). */
/* LB_Improved: LB_Keogh(x; L, U) + the query against the envelope of x
 * clamped into [L, U] (window r).  Squared. */
double orc_lb_improved2(const float *q, const double *U, const double *L, const float *x, int n, int r);
double orc_dtw2(const float *q, const float *x, int n, int r);

/* Exact k-NN by brute force (problem statement, Sec. 2.1; k-NN as a sorted
 * array of the k best, Sec. 5.4).  For every query, the k rows of data with
 * the smallest squared distance, ordered by (d2, id) ascending; ids are
 * id_base + row.  dist: 0 = ED, 1 = DTW with window r.  Outputs ids[nq*k],
 * d2[nq*k] (squared, FP64).  threads <= 0 means "all available". */
void orc_knn(const float *data, int64_t N, int n, const float *queries, int nq,
             int k, int dist, int r, int64_t id_base, int threads,
             int64_t *ids, double *d2);

/* Number of OpenMP threads the oracle would use for threads <= 0. */
int orc_max_threads(void);

/* Sliding-window subsequences (Sec. 2: a streaming series is cut into
 * subsequences of length n by a sliding window, which are then indexed;
 * Sec. 6: subsequence matching indexes every window of the query's length).
 * Window i = series[i*stride .. i*stride + n) for i < count =
 * (length - n) / stride + 1, written as row i of out.  With znorm each window
 * is z-normalised (mean 0, standard deviation 1, Sec. 2): mean = sequential
 * FP64 sum / n, var = sequential FP64 sum of (x - mean)^2 / n, inv =
 * 1 / sqrt(var) (0 when var is 0), out = (float)((x - mean) * inv).
 * Returns count. */
int64_t orc_windows(const float *series, int64_t length, int n, int stride, int znorm, float *out);

#ifdef __cplusplus
}
#endif
#endif
