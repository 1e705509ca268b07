/*
 * Measurement helpers of the AHPP library: device rates that roofline
 * reports divide by.  None of them touches a graph or a query; they live in
 * the same shared library as the query API (include/ahpp.h), whose status
 * codes they return.
 */
#ifndef AHPP_MEASURE_H
#define AHPP_MEASURE_H

#include "ahpp.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Row-access peak of a device, for roofline reporting (no graph needed).
 * The batched kernel moves its data as random 128-byte rows (32 queries x
 * FP32 of one node); once a table fits in L2 the L2 -> SM path, not HBM,
 * bounds those accesses.  This measures the rate, in rows per second, of
 * random 128-byte row gathers from (op 0) or float4 row reductions into
 * (op 1) a zero-filled device table of table_bytes (rounded down to 128-byte
 * rows), best of five launches after a warm-up.  Allocates and frees the
 * table itself and restores the caller's current device.  AHPP_EINVAL for
 * op not 0/1, table_bytes outside [128, 8 GiB], device < 0 or a NULL output;
 * AHPP_ENOMEM if the table cannot be allocated; AHPP_ECUDA otherwise. */
int ahpp_row_access_peak(int device, uint64_t table_bytes, int op, double *rows_per_s);

#ifdef __cplusplus
}
#endif

#endif /* AHPP_MEASURE_H */
