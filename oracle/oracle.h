/* Declarations shared by the oracle's C files (test infrastructure only). */
#ifndef ORACLE_H
#define ORACLE_H
#include <stdint.h>

typedef struct {
    int32_t m, n;
    int64_t nnz;
    int64_t *row_ptr;
    int32_t *col;
    double *val;
    double *g;
    uint8_t *is_int;
    int64_t *col_ptr;
    int32_t *row_idx;
    double *col_val;
} orc_problem;

typedef struct {
    int32_t status;
    int32_t rounds;
    int32_t first_infeasible_row;
    int32_t first_infeasible_var;
    int64_t nnz_updates;
    int64_t n_changed;
    int64_t candidates;
    int64_t fragile;
} orc_bp_result;

enum { ORC_FIXPOINT = 0, ORC_INFEASIBLE = 1, ORC_ROUND_LIMIT = 2 };

int orc_bp(const orc_problem *p, double *lb, double *ub, double *dlb, double *dub, const int32_t *w0, int32_t w0_len,
           double theta, int32_t max_rounds, int32_t mode, orc_bp_result *res, int64_t *trace_rows,
           int64_t *trace_nnz);
void orc_normalize(const orc_problem *p, double *lb, double *ub);
int orc_probe_split(int32_t is_int, double l, double u, double *out4);

#endif
