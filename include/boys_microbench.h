/*
 * boys_microbench.h -- throughput microbenchmarks used to build the ALU
 * roofline of the Boys kernels (how fast this GPU retires each FP64/FP32
 * operation the method of Sec. 2 uses: fused multiply-add, exponential,
 * square root, reciprocal square root, division).  Not part of the
 * evaluation path; the paper has no counterpart.
 */
#ifndef BOYS_GB300_MICROBENCH_H
#define BOYS_GB300_MICROBENCH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    BOYS_MICRO_DFMA = 0,  /* double fma */
    BOYS_MICRO_DEXP = 1,  /* double exp (plus one add) */
    BOYS_MICRO_DSQRT = 2, /* double sqrt (plus one add) */
    BOYS_MICRO_DRSQRT = 3,/* double rsqrt (plus one add) */
    BOYS_MICRO_DDIV = 4,  /* double division (plus one add) */
    BOYS_MICRO_FFMA = 5,  /* float fma */
    BOYS_MICRO_FEXP2 = 6, /* float exp2f (plus one add) */
    BOYS_MICRO_FSQRT = 7, /* float sqrtf (plus one add) */
    BOYS_MICRO_FDIV = 8,  /* float division (plus one add) */
    BOYS_MICRO_FRSQRT = 9,/* float rsqrtf (plus one add) */
    BOYS_MICRO_DEXP_LIB = 10 /* the library's own e^{-x} (Tang's method), plus one add */
};

/* Launch `blocks` x 256 threads, each running `iters` iterations of
 * boys_microbench_ops_per_thread_iter() independent operations of kind `op`
 * on `stream` (a cudaStream_t as void*).  `sink` is a device double that is
 * never actually written.  Returns a boys_status. */
int boys_microbench_launch(int op, int64_t iters, double *sink, int blocks, void *stream);

/* Independent operations per thread and iteration (the chain count). */
int boys_microbench_ops_per_thread_iter(void);

/* Double fused multiply-adds only, with `chains` independent chains per
 * thread (1, 2, 4, 8 or 16; anything else returns BOYS_ERR_ARG): `blocks` x
 * 256 threads, each running `iters` x `chains` fma on `stream`.  Sweeping
 * chains and blocks shows whether the DFMA rate of boys_microbench_launch is
 * the GPU's ceiling rather than a latency limit.  Returns a boys_status. */
int boys_microbench_dfma(int chains, int64_t iters, double *sink, int blocks, void *stream);

/* Integer-pipe kinds for boys_microbench_int.  The downward recursion and the
 * asymptote's chain of the double path run on 64-bit integer significands
 * (32 x 32 -> 64-bit multiply-adds, 64-bit adds and shifts); these measure
 * how fast the GPU retires such instructions, for a ceiling that counts the
 * integer pipes beside the FP64 pipe. */
enum {
    BOYS_MICRO_INT_MADWIDE = 0, /* mad.wide.u32: 32 x 32 -> 64-bit multiply-add */
    BOYS_MICRO_INT_MADLO = 1,   /* mad.lo.u32: 32-bit multiply-add */
    BOYS_MICRO_INT_ALU = 2,     /* add.u32 then xor.b32 (two instructions per chain step) */
    BOYS_MICRO_INT_SHIFT64 = 3  /* 64-bit shift by a run-time amount, then a 64-bit or */
};

/* Launch `blocks` x 256 threads, each running `iters` steps of 8 independent
 * chains of integer kind `kind` (BOYS_MICRO_INT_*) on `stream`.  `sink` is a
 * device double, written only if a 64-bit checksum of the chains takes one
 * particular value (in practice never).  Returns a boys_status
 * (BOYS_ERR_ARG for an unknown kind). */
int boys_microbench_int(int kind, int64_t iters, double *sink, int blocks, void *stream);

/* PTX instructions per chain step of an integer kind (-1 if unknown); the
 * pipe each one lands on is measured, not assumed. */
int boys_microbench_int_insts_per_chain_iter(int kind);

/* out[i] = e^{-x[i]} by the library's own exponential (Tang's table-driven
 * method), for testing it against a reference; valid for 0 <= x <= 700.
 * x, out: device arrays of n doubles.  Returns a boys_status. */
int boys_debug_exp_neg(const double *x, int64_t n, double *out, void *stream);

#ifdef __cplusplus
}
#endif

#endif
