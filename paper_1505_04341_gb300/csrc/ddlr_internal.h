// ddlr_internal.h -- entry points shared between the translation units of the
// library (not part of the C ABI).
#pragma once
#include "ddlr.h"

// batched PCG of R host right-hand sides (column-major n x R, leading dimension
// n) into host x, always through the batched kernels (also for R = 1), so a
// column's result does not depend on the other columns of its batch
ddlr_status pcg_batched_host(ddlr_handle h, const double *b, double *x, int R, double tol,
                             int maxit, ddlr_solve_info *info);
