// Host-side helpers shared by the library's translation units.
#pragma once
#include "ltjk_internal.h"

namespace ltjk {

int set_error(int code, const char *fmt, ...);
const char *last_error();

void normalise_shell(int l, int np, const double *exps, const double *coefs, double *out);
void boys_table(int rows, int cols, double step, double *tab);
int laplace_quadrature(double xmin, double xmax, int n, double *t_out, double *w_out,
                       double *err_out);
int laplace_minimax(double xmin, double xmax, int n, double *t_out, double *w_out,
                    double *err_out, int *converged);

}  // namespace ltjk
