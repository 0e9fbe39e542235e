// vc_aaa.cu -- the AAA multichannel timer update of Section II (Algorithm 1, Eqs. 1-9): per
// synchronisation interval (SI), the RSU folds the BSM statistics of the vehicles in its
// range into running values S_V2V (BSMs sent) and D_V2V (end-to-end delay per received
// BSM); at every UTC second it sets the effective CCH utilisation U_CCH = S_V2V * D_V2V and
// shortens the CCH interval to it (extending the SCH interval by the inactivity
// I_CCH = CCHI - U_CCH) when U_CCH is below the default CCHI, or restores the defaults.
// The SCHI fraction f = SCHI / SI it yields is the phase-flip parameter of the placement
// MDP.  Host code: a sequential recursion over a trace, O(SIs x vehicles).
#include <math.h>

#include "vc_internal.cuh"

using namespace vc;

extern "C" {

int vc_aaa_intervals(const double* S_v, const double* D_v, const double* R_v, int32_t n_vehicles, int32_t n_si,
                     int32_t si_per_second, double si_ms, double dcchi_ms, double dschi_ms, double* cchi_out,
                     double* schi_out, double* f_out) {
    set_error("");
    if (!S_v || !D_v || !R_v || !cchi_out || !schi_out) return fail(VC_ERR_ARG, "NULL argument");
    if (n_vehicles < 1 || n_si < 1 || si_per_second < 1) return fail(VC_ERR_ARG, "sizes must be >= 1");
    if (!(si_ms > 0.0) || !(dcchi_ms >= 0.0) || !(dschi_ms >= 0.0) || fabs(dcchi_ms + dschi_ms - si_ms) > 1e-9 * si_ms)
        return fail(VC_ERR_ARG, "the default intervals must be >= 0 and sum to the SI");
    double cchi = dcchi_ms, schi = dschi_ms;  // the intervals in force (IEEE 1609.4 defaults)
    double s_v2v = 0.0, d_v2v = 0.0;          // running BSM count and delay of the current second
    int64_t out = 0;
    for (int32_t j = 0; j < n_si; j++) {
        const double* S = S_v + (int64_t)j * n_vehicles;
        const double* D = D_v + (int64_t)j * n_vehicles;
        const double* R = R_v + (int64_t)j * n_vehicles;
        if ((j + 1) % si_per_second != 0) {
            // not the UTC second: fold this SI's statistics in (Algorithm 1, lines 5-6)
            double ss = 0.0, ds = 0.0, rs = 0.0;
            for (int32_t h = 0; h < n_vehicles; h++) {
                ss += S[h];
                ds += D[h];
                rs += R[h];
            }
            s_v2v = (s_v2v + ss) / (1.0 + n_vehicles);
            d_v2v = (d_v2v + ds) / (1.0 + rs);
        } else {
            // the UTC second: effective utilisation and inactivity (Eqs. 4, 7), then the
            // timer update (Eq. 8) or the reset to the defaults
            const double u_cch = s_v2v * d_v2v;
            const double i_cch = cchi - u_cch;
            if (u_cch < dcchi_ms) {
                cchi = u_cch;
                schi = schi + i_cch;
            } else {
                cchi = dcchi_ms;
                schi = dschi_ms;
            }
            cchi_out[out] = cchi;
            schi_out[out] = schi;
            if (f_out) f_out[out] = schi / si_ms;
            out++;
            s_v2v = 0.0;
            d_v2v = 0.0;
        }
    }
    return VC_OK;
}

}  // extern "C"
