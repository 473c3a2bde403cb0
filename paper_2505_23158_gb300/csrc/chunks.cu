// Chunk centres from camera positions (supplementary "Selecting chunk
// centers"): the number of clusters of Eq. 5 and K-means (Lloyd) on the
// training camera positions.  A load-time step over at most a few thousand
// positions, done on the host in FP64 with a fixed order of operations
// (distances as (dx*dx + dy*dy) + dz*dz, member sums in index order; the
// library is compiled without floating-point contraction) so that results
// are reproducible bit for bit.
#include <cmath>
#include <vector>

#include "internal.cuh"

namespace lodge {
namespace {

double dist2(const double* a, const double* b) {
    const double dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
    return (dx * dx + dy * dy) + dz * dz;
}

// nearest of k centres (squared Euclidean), ties to the lower index
int32_t nearest(const double* p, const double* m, int32_t k) {
    int32_t best = 0;
    double bd = dist2(p, m);
    for (int32_t j = 1; j < k; ++j) {
        const double d = dist2(p, m + 3 * j);
        if (d < bd) { bd = d; best = j; }
    }
    return best;
}

}  // namespace
}  // namespace lodge

using namespace lodge;

extern "C" lodge_status lodge_num_clusters(const double* positions, int32_t n, double d1,
                                           int32_t* k_out) {
    if (!positions || n < 1 || !k_out || !(d1 > 0.0) || !std::isfinite(d1))
        return set_error(LODGE_E_INVALID, "bad argument");
    double mean[3] = {0.0, 0.0, 0.0};
    for (int32_t i = 0; i < n; ++i)
        for (int c = 0; c < 3; ++c) mean[c] += positions[3 * i + c];
    for (int c = 0; c < 3; ++c) mean[c] /= (double)n;
    double rmax = 0.0;
    for (int32_t i = 0; i < n; ++i) {
        const double r = std::sqrt(dist2(positions + 3 * i, mean));
        if (r > rmax) rmax = r;
    }
    const double k = std::ceil(4.0 / d1 * rmax);
    int32_t kk = k < 1.0 ? 1 : (k > (double)n ? n : (int32_t)k);
    *k_out = kk;
    return LODGE_OK;
}

extern "C" lodge_status lodge_kmeans_centers(const double* positions, int32_t n, int32_t k,
                                             const int32_t* init, int32_t max_iter,
                                             double* centers_out, int32_t* assign_out,
                                             int32_t* iters_out) {
    if (!positions || !init || !centers_out || n < 1 || k < 1 || k > n || max_iter < 0)
        return set_error(LODGE_E_INVALID, "bad argument");
    std::vector<double> m((size_t)3 * k);
    for (int32_t j = 0; j < k; ++j) {
        if (init[j] < 0 || init[j] >= n) return set_error(LODGE_E_INVALID, "initial index out of range");
        for (int32_t i = 0; i < j; ++i)
            if (init[i] == init[j]) return set_error(LODGE_E_INVALID, "initial indices must be distinct");
        for (int c = 0; c < 3; ++c) m[3 * j + c] = positions[3 * init[j] + c];
    }
    std::vector<int32_t> a((size_t)n, -1);
    std::vector<double> sum((size_t)3 * k);
    std::vector<int64_t> cnt((size_t)k);
    int32_t it = 0;
    for (; it < max_iter; ++it) {
        // assignment: nearest centre, ties to the lower index
        bool changed = false;
        for (int32_t i = 0; i < n; ++i) {
            const int32_t best = nearest(positions + 3 * i, m.data(), k);
            if (a[i] != best) { a[i] = best; changed = true; }
        }
        if (!changed) break;
        // update: mean of the members, summed in index order
        std::fill(sum.begin(), sum.end(), 0.0);
        std::fill(cnt.begin(), cnt.end(), 0);
        for (int32_t i = 0; i < n; ++i) {
            for (int c = 0; c < 3; ++c) sum[3 * a[i] + c] += positions[3 * i + c];
            ++cnt[a[i]];
        }
        for (int32_t j = 0; j < k; ++j)
            if (cnt[j])
                for (int c = 0; c < 3; ++c) m[3 * j + c] = sum[3 * j + c] / (double)cnt[j];
    }
    for (size_t i = 0; i < m.size(); ++i) centers_out[i] = m[i];
    if (assign_out)   // nearest returned centre of every position
        for (int32_t i = 0; i < n; ++i) assign_out[i] = nearest(positions + 3 * i, m.data(), k);
    if (iters_out) *iters_out = it;
    return LODGE_OK;
}
