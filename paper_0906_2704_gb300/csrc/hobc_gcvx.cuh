// Shared parts of the GCV curve by bin expansion (hobc_gcvx.cu: plans;
// hobc_batched.cu: batches): the bin geometry, the classification of an entry,
// the per-key terms of the curve and float-float accumulation.  The method is
// described in hobc_gcvx.cu.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstring>

#include "hobc_kernels.cuh"

namespace hobc {

static const int kGxBins = 256;               // inner bins, uniform in log a
static const int kGxKeys = kGxBins + 2;       // key 0: a < a_lo; 1..256 inner; 257: a >= a_hi
static const int kGxP = 8;                    // moments p = 0..7

struct GxTab {                                // bin geometry (device copy)
    float abar[kGxBins];                      // bin centres a_lo r^(b + 1/2)
    float inv_abar[kGxBins];
    float edge[kGxBins + 1];                  // bin edges a_lo r^b
    float a_lo, a_hi, inv_alo;
    float log2_alo, bins_per_log2;            // b = floor((log2 a - log2 a_lo) bins_per_log2)
};

// Truncation bound of the series for a grid [mu_min, mu_max] (relative error of
// a numerator term; the denominator's is smaller): 9 U^8/(1-U)^2 with U the
// largest |rho u| of an inner bin (and 9 (1e-3)^8 for the outer keys).
inline double gx_bound(double mu_min, double mu_max, double* r_out) {
    const double decades = std::log10(mu_max / mu_min) + 6.0;
    const double r = std::pow(10.0, decades / kGxBins);
    const double U = std::sqrt(r) - 1.0 + 1e-6;             // margin for the rounding of the edges
    if (r_out) *r_out = r;
    return std::max(9.0 * std::pow(U, 8) / ((1 - U) * (1 - U)), 9.0 * std::pow(1e-3, 8));
}

// The bin geometry of a grid of K positive values; its bound in *bound.
inline void gx_make_table(const double* mu, int K, GxTab& t, double* bound) {
    const double mu_min = *std::min_element(mu, mu + K), mu_max = *std::max_element(mu, mu + K);
    double r = 0;
    *bound = gx_bound(mu_min, mu_max, &r);
    memset(&t, 0, sizeof(t));
    const double a_lo = 1e-3 * mu_min;
    for (int b = 0; b <= kGxBins; ++b) t.edge[b] = (float)(a_lo * std::pow(r, b));
    for (int b = 0; b < kGxBins; ++b) {
        const double ab = a_lo * std::pow(r, b + 0.5);
        t.abar[b] = (float)ab;
        t.inv_abar[b] = (float)(1.0 / ab);
    }
    t.a_lo = (float)a_lo;
    t.a_hi = t.edge[kGxBins];
    t.inv_alo = (float)(1.0 / a_lo);
    t.log2_alo = (float)std::log2(a_lo);
    t.bins_per_log2 = (float)(1.0 / std::log2(r));
}

// float-float accumulation: hi + lo += x, with the rounding error of hi + x kept
// in lo (TwoSum; the _rn intrinsics keep the compiler from fusing or reordering)
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x) {
    const float s = __fadd_rn(hi, x);
    const float bv = __fsub_rn(s, hi);
    lo += __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bv)), __fsub_rn(x, bv));
    hi = s;
}

// The key of an entry with a = |d|^2/|s|^2 (capped) and weight w, its expansion
// coordinate u and the scales of its numerator and denominator terms.  Branch
// free: the inner bin is found for every a (clamped) and the outer keys chosen
// by selects; 1/a is one correctly rounded reciprocal (key 257: u = a_hi/a,
// w/a, w/a^2).
__device__ __forceinline__ int gx_classify(float a, float w, const GxTab* __restrict__ tab, float& u, float& vn,
                                           float& vd) {
    int b = (int)floorf((__log2f(a) - tab->log2_alo) * tab->bins_per_log2);
    b = max(0, min(kGxBins - 1, b));
    if (a < tab->edge[b] && b > 0) --b;                         // the approximate log2 may be one bin off
    else if (a >= tab->edge[b + 1] && b < kGxBins - 1) ++b;
    const float ub = (a - tab->abar[b]) * tab->inv_abar[b];
    const bool small = a < tab->a_lo, large = a >= tab->a_hi;
    const float ra = __frcp_rn(large ? a : 1.f);
    u = small ? a * tab->inv_alo : (large ? tab->a_hi * ra : ub);
    vd = large ? w * ra : w;
    vn = large ? vd * ra : w;
    return small ? 0 : (large ? kGxKeys - 1 : 1 + b);
}

// The factors of key k at grid value m: the series variable x and the scales of
// the numerator and denominator sums (1/(abar+m)^2 and 1/(abar+m) for the inner
// bins).
__device__ __forceinline__ void gx_key_terms(int k, float m, const GxTab* __restrict__ tab, float& x, float& sn,
                                             float& sd) {
    if (k == 0) {
        const float inv = __fdividef(1.f, m);
        x = -tab->a_lo * inv; sn = inv * inv; sd = inv;
    } else if (k == kGxKeys - 1) {
        x = -m / tab->a_hi; sn = 1.f; sd = 1.f;
    } else {
        const float ab = tab->abar[k - 1];
        const float inv = __fdividef(1.f, ab + m);
        x = -ab * inv; sn = inv * inv; sd = inv;
    }
}

}  // namespace hobc
