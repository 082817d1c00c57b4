// Host-only evaluation of the near-field blob series with the kernels' own
// coefficient table (make_series): prints rho, q = g/rho^3 and f = F/rho^5 in
// double arithmetic, for comparison with the FP64 oracle.
#include <math.h>
#include <stdio.h>

#include "vpm_kernel.cuh"

int main()
{
    const vpm::SeriesCoef s = vpm::make_series();
    const double rhos[] = {1e-3, 0.05, 0.3, 0.7, 1.0, 1.4, 1.8, 1.99};
    for (double rho : rhos) {
        const double x = 0.5 * rho * rho;
        double T = s.c[15], U = s.d[15];
        for (int k = 14; k >= 0; --k) {
            T = T * x + s.c[k];
            U = U * x + s.d[k];
        }
        const double e = exp(-x) * pow(2.0, -1.5);
        printf("%.17g %.17g %.17g\n", rho, e * T, -e * U);
    }
    return 0;
}
