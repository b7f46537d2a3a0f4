/*
 * mdp_probe.h -- measurement utility of libmdp: the FP64 fused multiply-add throughput of
 * the current CUDA device, the denominator of the FP64 roofline of the projection kernels.
 * (No counterpart in the paper, which reports no hardware figures.)
 */
#ifndef MDP_PROBE_H
#define MDP_PROBE_H
#include "mdp.h"
#ifdef __cplusplus
extern "C" {
#endif

/* Runs a DFMA microbenchmark (8 independent chains per thread, 8 resident blocks of 256
 * threads per SM, `iters` iterations; 0 selects 4096) on `cuda_stream`, synchronises and
 * writes the achieved FP64 GFLOP/s (2 flops per DFMA) to *gflops (host). Allocates and frees
 * a small device buffer. Returns MDP_ERR_CUDA on a CUDA failure. */
mdp_status mdp_probe_dfma_gflops(int iters, double *gflops, void *cuda_stream);

/* The same for the FP64 tensor-core path: 8 independent chains of mma.sync m8n8k4 FP64 MMAs
 * (512 flops each) per warp, 8 resident blocks of 256 threads per SM, `iters` iterations (0
 * selects 2048). Writes the achieved FP64 GFLOP/s. It decides whether a dense FP64 contraction
 * of the path belongs on the tensor cores or on the FMA pipe (no counterpart in the paper). */
mdp_status mdp_probe_dmma_gflops(int iters, double *gflops, void *cuda_stream);

/* Per-kernel timing of a plan's launches (tracing). enable = 1 starts recording a CUDA event
 * pair around every kernel launch of mdp_project_batch / mdp_project_columns / mdp_ap_adjoint
 * on the launch stream (events are created on demand; no device memory is allocated);
 * enable = 0 stops. mdp_plan_profile_read synchronises the recorded events, returns the summed
 * duration (ms) and the number of launches of kernel family `family` since the last read, and
 * resets that family's record. Families are numbered 0..mdp_kernel_family_count()-1. */
mdp_status mdp_plan_profile(mdp_plan *p, int enable);
mdp_status mdp_plan_profile_read(mdp_plan *p, int family, double *total_ms, int *launches);
int mdp_kernel_family_count(void);
const char *mdp_kernel_family_name(int family);

/* Geometry of subdomain `sub` as 14 ints: Px, Py (M+ nodes per direction), Nq (sine modes),
 * Nt (tridiagonal rows), i0 (first swept row), nfirst (first unknown y row), complex factors
 * (0/1), |gamma|, |ring|, number of pivoted rows over all modes, n_cols, Nx, x-centred (0/1),
 * number of factor rows with complex entries swept by the projection, over all modes. */
mdp_status mdp_plan_sub_info(const mdp_plan *p, int sub, int *info14);

/* Bytes of the plan's tables (factors, sweep tables, sines, geometry, pivot flags), uploaded at
 * plan creation and rebuilt on the device by mdp_plan_update_k. */
long long mdp_plan_table_bytes(const mdp_plan *p);

/* Bytes that mdp_plan_update_k copies host -> device on a device plan (the subdomain
 * descriptors with the new wavenumbers; the tables themselves are rebuilt on the device). */
long long mdp_plan_update_bytes(const mdp_plan *p);

/* Sizes of the plan's tables: doubles (factor, dT/dk, sine, segment, sweep and geometry tables)
 * and pivot-flag bytes. */
mdp_status mdp_plan_table_sizes(const mdp_plan *p, long long *n_doubles, long long *n_piv);

/* Copy the tables into caller-owned host buffers of mdp_plan_table_sizes elements: the device
 * copy (device_side = 1; MDP_ERR_STATE on a host-only plan) or the host copy (device_side = 0,
 * rebuilt on the host for the current wavenumbers if the device has refactored since). Used to
 * check the device factorisation against the host one. */
mdp_status mdp_plan_read_tables(const mdp_plan *p, int device_side, double *tables, unsigned char *piv);

/* y[i] = 1/x[i] for x[i] > 0 (device arrays of n doubles, on cuda_stream) by the reciprocal
 * that the device factorisation uses: a single-precision seed refined by one cubic
 * Newton-Raphson (Goldschmidt) step; outside [2^-120, 2^120] a division. For testing its error
 * against 1/x. */
mdp_status mdp_probe_rcp(const double *x, double *y, int n, void *cuda_stream);

/* Offsets of subdomain `sub`'s tables (7 values): in doubles into the tables, the factor rows
 * [Nq][Nt][8 complex | 4 real AP], dT/dk rows [Nq][Nt][6], sines [4 Nx], segments [Nq][5],
 * sweep rows [Nq][rows from i0][24], gamma geometry [|gamma|][4]; then in bytes into the pivot
 * flags [Nq][Nt]. */
mdp_status mdp_plan_table_offsets(const mdp_plan *p, int sub, long long *off7);

#ifdef __cplusplus
}
#endif
#endif
