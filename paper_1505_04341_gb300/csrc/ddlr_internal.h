// ddlr_internal.h -- entry points shared between the translation units of the
// library (not part of the C ABI).
#pragma once
#include "ddlr.h"


// Continuous batching for the serving runtime: a block PCG of width R whose
// columns (slots) are admitted and retired between iterations; a column's
// iterates are those of its solve alone (ddlr_batch.cuh).  One thread per
// handle.
ddlr_status slots_open(ddlr_handle h, int R, double tol, int maxit);
// lay the open block out as R1 columns, new column q = old column map[q]
// (map[q] < 0: a new idle column); running columns continue unchanged
ddlr_status slots_resize(ddlr_handle h, int R1, const int *map);
// admit host right-hand sides b[i] (original order) into free slots slot[i]
ddlr_status slots_admit(ddlr_handle h, int cnt, const int *slot, const double *const *b);
// run `iters` iterations; done[q] (R ints) = 1 for finished or idle slots
ddlr_status slots_run(ddlr_handle h, int iters, int *done);
// copy out a finished slot's result (host x, original order); frees the slot
ddlr_status slots_take(ddlr_handle h, int slot, double *x, ddlr_solve_info *info);
int slots_width(ddlr_handle h);
void slots_forget(ddlr_handle h);
