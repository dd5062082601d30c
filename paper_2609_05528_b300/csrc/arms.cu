// Mechanism arms of Sec. 6.4 as ray-table transforms (host code).  The paper
// names the pairing-destroyed, delay-only and spatial-only controls without
// giving their construction; the readings implemented here are:
//  * pairing destroyed: within each order the delays are redistributed over
//    the order's rays by a permutation drawn from caller-supplied keys, so
//    each order keeps its delay multiset while the pairing of delay with
//    source point and weight is broken;
//  * delay-only: every ring ray (order >= 1) keeps its delay, weight and row
//    and takes the source point (r, phi) of its direct quantile partner;
//  * spatial-only: every ring ray keeps its source point, weight and row and
//    takes the delay of its direct quantile partner.
// The direct quantile partner of the ray of rank k (by delay, ties by index)
// among the E_n rays of order n is the direct ray of rank
// floor((k + 1/2) E_0 / E_n) among the E_0 direct rays.
#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "rtt_internal.cuh"

using namespace rtt;

namespace {

// ray indices of order n, ascending
std::vector<int64_t> rays_of_order(const rtt_ray_table* t, int n) {
    std::vector<int64_t> v;
    for (int64_t e = 0; e < t->n_rays; ++e)
        if (t->order[e] == n) v.push_back(e);
    return v;
}

// the same rays ranked by (value, index)
void rank_by(std::vector<int64_t>& v, const double* value) {
    std::stable_sort(v.begin(), v.end(), [value](int64_t a, int64_t b) {
        return value[a] < value[b] || (value[a] == value[b] && a < b);
    });
}

}  // namespace

extern "C" rtt_status rtt_arm_table(int kind, const rtt_ray_table* in, const double* keys_host,
                                    double* r_out, double* phi_out, double* delay_out) {
    if (!in || in->n_rays < 1 || !in->order || !in->r || !in->phi || !in->delay || !r_out ||
        !phi_out || !delay_out ||
        (kind != RTT_ARM_PAIRING_DESTROYED && kind != RTT_ARM_DELAY_ONLY &&
         kind != RTT_ARM_SPATIAL_ONLY) ||
        (kind == RTT_ARM_PAIRING_DESTROYED && !keys_host)) {
        set_error("rtt_arm_table: invalid arguments (kind %d)", kind);
        return RTT_EINVAL;
    }
    const int64_t E = in->n_rays;
    for (int64_t e = 0; e < E; ++e) {
        if (in->order[e] < 0 || in->order[e] > 2 || !std::isfinite(in->delay[e]) ||
            (keys_host && kind == RTT_ARM_PAIRING_DESTROYED && !std::isfinite(keys_host[e]))) {
            set_error("rtt_arm_table: ray %lld has an invalid order, delay or key", (long long)e);
            return RTT_EINVAL;
        }
    }
    try {
        std::vector<double> r(in->r, in->r + E), phi(in->phi, in->phi + E),
            delay(in->delay, in->delay + E);
        if (kind == RTT_ARM_PAIRING_DESTROYED) {
            for (int n = 0; n < 3; ++n) {
                const std::vector<int64_t> by_index = rays_of_order(in, n);
                std::vector<int64_t> by_key = by_index;
                rank_by(by_key, keys_host);
                for (size_t m = 0; m < by_index.size(); ++m) delay[by_index[m]] = in->delay[by_key[m]];
            }
        } else {
            std::vector<int64_t> direct = rays_of_order(in, 0);
            if (direct.empty()) {
                set_error("rtt_arm_table: the table has no direct ray");
                return RTT_EINVAL;
            }
            rank_by(direct, in->delay);
            const int64_t E0 = (int64_t)direct.size();
            for (int n = 1; n < 3; ++n) {
                std::vector<int64_t> ring = rays_of_order(in, n);
                rank_by(ring, in->delay);
                const int64_t En = (int64_t)ring.size();
                for (int64_t k = 0; k < En; ++k) {
                    const int64_t p = direct[((2 * k + 1) * E0) / (2 * En)];
                    const int64_t e = ring[k];
                    if (kind == RTT_ARM_DELAY_ONLY) {
                        r[e] = in->r[p];
                        phi[e] = in->phi[p];
                    } else {
                        delay[e] = in->delay[p];
                    }
                }
            }
        }
        std::copy(r.begin(), r.end(), r_out);
        std::copy(phi.begin(), phi.end(), phi_out);
        std::copy(delay.begin(), delay.end(), delay_out);
    } catch (const std::bad_alloc&) {
        set_error("rtt_arm_table: host allocation failed");
        return RTT_ENOMEM;
    }
    return RTT_OK;
}
