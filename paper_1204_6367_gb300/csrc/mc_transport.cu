// Monte Carlo photon transport, Section 2.4 of the paper, for sm_103a.
//
// One CUDA thread tracks one photon history at a time (as in the paper), but
// the grid is persistent: warps claim chunks of histories from a global
// counter and refill lanes whose history ended, so lanes stay busy while
// histories of very different lengths finish.  Tallies are int64 fixed point
// (2^-24 keV), summed with integer atomics, so the result does not depend on
// which lane ran which history or in which order.
//
// Arithmetic contract.  This file is compiled with -fmad=false: every FP32
// operation below is one IEEE-rounded operation, evaluated in the order
// written (divide and square root are the correctly rounded ones).  The only
// transcendental is the logarithm of the free-flight length, computed by the
// atanh series in gd_logf below.  Together with the counter-based random
// streams this makes a history's result a function of (seed, angle index,
// history id) alone.
//
// Readings of points the paper leaves open:
//  * random numbers: Philox4x32-10 (Salmon et al., SC'11), key = seed,
//    counter = (block, angle index, history id lo, hi); uniforms are
//    ((word >> 8) + 1) * 2^-24 in (0, 1];
//  * source: detector pixel from the fluence map w(u) and channel from the
//    spectrum phi(E), each by inverse CDF; uniform point inside the pixel;
//  * material at an off-centre point: per-material trilinear partial
//    densities, mu(x, E) = sum_m mu_hat(m, E) rho_m(x) (density interpolation
//    of Section 2.4, consistent with the ray-traced field of Section 2.3);
//  * field: clamp to edge inside the voxel box, vacuum outside;
//  * Woodcock majorant mu_max(E): largest mu over materials at their largest
//    density, the larger of the two bracketing energy nodes;
//  * Compton: free-electron Klein-Nishina by Kahn's rejection method;
//    Rayleigh: Thomson (1 + cos^2) by rejection; azimuth from a point of the
//    unit disc;
//  * tally: rint(r(E) * 2^24) into the primary counter when the photon never
//    scattered, else the scatter counter (Section 2.4).
#include "gdrr_internal.cuh"

namespace gdrr {
namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ void philox4x32_10(uint32_t& c0, uint32_t& c1, uint32_t& c2, uint32_t& c3,
                                              uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0;
        const uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

// The random stream of one history: words consumed in order, four per block.
struct Stream {
    uint32_t k0, k1, angle, hlo, hhi, blk;
    uint32_t b0, b1, b2, b3;
    int pos;

    __device__ __forceinline__ void init(uint64_t seed, uint32_t angle_index, uint64_t hid) {
        k0 = (uint32_t)seed; k1 = (uint32_t)(seed >> 32);
        angle = angle_index; hlo = (uint32_t)hid; hhi = (uint32_t)(hid >> 32);
        blk = 0; pos = 4;
    }
    __device__ __forceinline__ uint32_t word() {
        if (pos == 4) {
            uint32_t c0 = blk, c1 = angle, c2 = hlo, c3 = hhi;
            philox4x32_10(c0, c1, c2, c3, k0, k1);
            b0 = c0; b1 = c1; b2 = c2; b3 = c3;
            ++blk;
            pos = 0;
        }
        const uint32_t w = pos == 0 ? b0 : (pos == 1 ? b1 : (pos == 2 ? b2 : b3));
        ++pos;
        return w;
    }
    __device__ __forceinline__ float uniform() {
        return (float)((word() >> 8) + 1u) * (float)(1.0 / 16777216.0);
    }
};

// ln(x), x a positive normal float: x = m 2^e, m in [sqrt(1/2), sqrt(2)),
// ln m = 2 atanh(s), s = (m - 1)/(m + 1), by the Taylor series of atanh to
// s^11 (|s| <= 0.1716, remainder below 2^-30), ln 2 split into a 12-bit head
// (exact products with e) and a tail.
__device__ __forceinline__ float gd_logf(float x) {
    uint32_t u = __float_as_uint(x);
    int e = (int)((u >> 23) & 0xffu) - 127;
    u = (u & 0x007fffffu) | 0x3f800000u;
    if (u > 0x3fb504f3u) {
        u -= 0x00800000u;
        e += 1;
    }
    const float m = __uint_as_float(u);
    const float s = (m - 1.0f) / (m + 1.0f);
    const float s2 = s * s;
    const float poly = (float)(1.0 / 3.0) + s2 * ((float)(1.0 / 5.0) + s2 * ((float)(1.0 / 7.0)
                     + s2 * ((float)(1.0 / 9.0) + s2 * (float)(1.0 / 11.0))));
    const float lm = 2.0f * s + (2.0f * s) * (s2 * poly);
    const float fe = (float)e;
    return fe * (float)(2839.0 / 4096.0) + (fe * (float)(0.69314718055994530942 - 2839.0 / 4096.0) + lm);
}

// Smallest j with xi <= cdf[j]; the guide table gives a start, two short scans finish.
__device__ __forceinline__ int cdf_search(const double* __restrict__ cdf, const int* __restrict__ guide,
                                          int n_guide, double xi) {
    int gi = (int)(xi * (double)n_guide);
    gi = gi < 0 ? 0 : (gi > n_guide - 1 ? n_guide - 1 : gi);
    int j = __ldg(guide + gi);
    while (j > 0 && xi <= __ldg(cdf + j - 1)) --j;
    while (xi > __ldg(cdf + j)) ++j;
    return j;
}

__device__ __forceinline__ void interp_index(float e, float e0, float inv_de, int n, int& i, float& f) {
    float fi = (e - e0) * inv_de;
    if (fi < 0.0f) fi = 0.0f;
    if (fi > (float)(n - 1)) fi = (float)(n - 1);
    int ie = (int)fi;
    if (ie > n - 2) ie = n - 2;
    i = ie;
    f = fi - (float)ie;
}

template <int NM>
struct Coeffs {
    float r[NM], c[NM], p[NM];
    float mumax;

    __device__ __forceinline__ void at(const McParams& P, float e) {
        int ie; float f;
        interp_index(e, P.e0, P.inv_de, P.n_e, ie, f);
#pragma unroll
        for (int m = 0; m < NM; ++m) {
            if (m < P.n_mat) {
                const float* t = P.tab + (size_t)m * 3 * P.n_e;
                const float r0 = __ldg(t + ie), r1 = __ldg(t + ie + 1);
                const float c0 = __ldg(t + P.n_e + ie), c1 = __ldg(t + P.n_e + ie + 1);
                const float p0 = __ldg(t + 2 * P.n_e + ie), p1 = __ldg(t + 2 * P.n_e + ie + 1);
                r[m] = r0 + f * (r1 - r0);
                c[m] = c0 + f * (c1 - c0);
                p[m] = p0 + f * (p1 - p0);
            } else {
                r[m] = 0.0f; c[m] = 0.0f; p[m] = 0.0f;
            }
        }
        const float a = __ldg(P.major + ie), b = __ldg(P.major + ie + 1);
        mumax = a > b ? a : b;
    }
};

__device__ __forceinline__ float response(const McParams& P, float e) {
    int ir; float f;
    interp_index(e, P.r0, P.inv_dr, P.n_r, ir, f);
    const float a = __ldg(P.resp + ir), b = __ldg(P.resp + ir + 1);
    return a + f * (b - a);
}

__device__ __forceinline__ void azimuth(Stream& rs, float& cp, float& sp) {
    for (;;) {
        const float a = 2.0f * rs.uniform() - 1.0f;
        const float b = 2.0f * rs.uniform() - 1.0f;
        const float r2 = a * a + b * b;
        if (r2 <= 1.0f && r2 > 0.0f) {
            cp = (a * a - b * b) / r2;
            sp = 2.0f * a * b / r2;
            return;
        }
    }
}

__device__ __forceinline__ void rotate(float& u, float& v, float& w, float ct, float cp, float sp) {
    const float st2 = 1.0f - ct * ct;
    const float st = st2 > 0.0f ? sqrtf(st2) : 0.0f;
    float nu_, nv_, nw_;
    if (w < (float)0.99999 && w > (float)-0.99999) {
        const float t = sqrtf(1.0f - w * w);
        nu_ = u * ct + st * (u * w * cp - v * sp) / t;
        nv_ = v * ct + st * (v * w * cp + u * sp) / t;
        nw_ = w * ct - st * t * cp;
    } else {
        nu_ = st * cp;
        nv_ = st * sp;
        nw_ = w > 0.0f ? ct : -ct;
    }
    const float len = sqrtf(nu_ * nu_ + nv_ * nv_ + nw_ * nw_);
    u = nu_ / len;
    v = nv_ / len;
    w = nw_ / len;
}

__device__ __forceinline__ void compton(Stream& rs, float e, float& ct_out, float& e_out) {
    const float alpha = e / (float)510.99895;
    const float ta = 2.0f * alpha;
    float x;
    for (;;) {
        const float r1 = rs.uniform();
        const float r2 = rs.uniform();
        const float r3 = rs.uniform();
        if (r1 <= (1.0f + ta) / (9.0f + ta)) {
            x = 1.0f + ta * r2;
            if (r3 <= 4.0f * (x - 1.0f) / (x * x)) break;
        } else {
            x = (1.0f + ta) / (1.0f + ta * r2);
            const float ct = 1.0f - (x - 1.0f) / alpha;
            if (r3 <= 0.5f * (ct * ct + 1.0f / x)) break;
        }
    }
    ct_out = 1.0f - (x - 1.0f) / alpha;
    e_out = e / x;
}

__device__ __forceinline__ float rayleigh(Stream& rs) {
    for (;;) {
        const float a = rs.uniform();
        const float b = rs.uniform();
        const float mu = 2.0f * a - 1.0f;
        if (2.0f * b <= 1.0f + mu * mu) return mu;
    }
}

enum : uint32_t { OUT_PRIMARY = 0, OUT_SCATTER = 1, OUT_PHOTO = 2, OUT_CUTOFF = 3, OUT_MISS = 4, OUT_STEP_LIMIT = 5 };

// Per-lane counters, summed into the stats array when the lane retires.
struct Counters {
    uint32_t hist, steps, virt, ray, comp, photo, tp, ts, miss, cut, lim;
};

template <int NM, bool REC>
struct Lane {
    // photon state
    float px, py, pz, dx, dy, dz, e;
    int scattered;
    int job;
    uint64_t gidx;
    uint32_t nsteps;
    Stream rs;
    Coeffs<NM> co;
    // event record (REC only)
    uint32_t r_virt, r_ray, r_comp, r_first;
    float r_esrc;
    double r_dep;

    __device__ __forceinline__ void record(const McParams& P, uint32_t outcome, int pixel, uint32_t photo) {
        if (!REC) return;
        gdrr_history_record r;
        r.n_steps = nsteps; r.n_virtual = r_virt; r.n_rayleigh = r_ray; r.n_compton = r_comp;
        r.n_photo = photo; r.outcome = outcome; r.rng_blocks = rs.blk; r.first_interaction = r_first;
        r.pixel = pixel; r.e_source = r_esrc; r.e_final = e; r.pad = 0; r.e_deposited = r_dep;
        P.records[gidx] = r;
    }

    // The photon left the phantom (or never entered it): straight line to
    // the imager plane, tally r(E) at the pixel it meets.
    __device__ __forceinline__ void escape(const McParams& P, Counters& k) {
        const Job& J = P.jobs[job];
        const float n0 = J.f.n[0], n1 = J.f.n[1], n2 = J.f.n[2];
        const float dn = dx * n0 + dy * n1 + dz * n2;
        uint32_t outcome = OUT_MISS;
        int pixel = -1;
        if (dn > 0.0f) {
            const float P0 = J.f.P[0], P1 = J.f.P[1], P2 = J.f.P[2];
            const float num = (P0 - px) * n0 + (P1 - py) * n1 + (P2 - pz) * n2;
            const float tt = num / dn;
            if (tt >= 0.0f) {
                const float rel0 = (px + tt * dx) - P0;
                const float rel1 = (py + tt * dy) - P1;
                const float rel2 = (pz + tt * dz) - P2;
                const float au = rel0 * J.f.eu[0] + rel1 * J.f.eu[1] + rel2 * J.f.eu[2];
                const float av = rel0 * J.f.ev[0] + rel1 * J.f.ev[1] + rel2 * J.f.ev[2];
                const float fu = au * P.idu + P.hu;
                const float fv = av * P.idv + P.hv;
                if (fu >= 0.0f && fu < (float)P.nu && fv >= 0.0f && fv < (float)P.nv) {
                    pixel = (int)fv * P.nu + (int)fu;
                    const long long q = llrintf(response(P, e) * 16777216.0f);
                    int64_t* t = scattered ? J.tally_s : J.tally_p;
                    atomicAdd(reinterpret_cast<unsigned long long*>(t + pixel), (unsigned long long)q);
                    outcome = scattered ? OUT_SCATTER : OUT_PRIMARY;
                }
            }
        }
        if (outcome == OUT_PRIMARY) ++k.tp;
        else if (outcome == OUT_SCATTER) ++k.ts;
        else ++k.miss;
        record(P, outcome, pixel, 0);
    }

    __device__ __forceinline__ void move_to_box_exit(const McParams& P) {
        float te = (float)3.0e38;
        const float d[3] = {dx, dy, dz};
        const float p[3] = {px, py, pz};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (d[a] > 0.0f) {
                const float t = (P.hi[a] - p[a]) / d[a];
                if (t < te) te = t;
            } else if (d[a] < 0.0f) {
                const float t = (P.lo[a] - p[a]) / d[a];
                if (t < te) te = t;
            }
        }
        if (te < 0.0f) te = 0.0f;
        px = px + te * dx;
        py = py + te * dy;
        pz = pz + te * dz;
    }

    // Start history gidx; returns true when it is still in flight.
    __device__ __forceinline__ bool start(const McParams& P, uint64_t g, Counters& k) {
        gidx = g;
        int lo = 0, hi = P.n_jobs - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (P.jobs[mid].first <= g) lo = mid; else hi = mid - 1;
        }
        job = lo;
        const Job& J = P.jobs[job];
        const uint64_t hid = J.hid_offset + (g - J.first);
        rs.init(P.seed, J.angle_index, hid);
        ++k.hist;
        nsteps = 0;
        scattered = 0;
        if (REC) { r_virt = 0; r_ray = 0; r_comp = 0; r_first = 0; r_dep = 0.0; }

        const float xi_pix = rs.uniform();
        const float xi_u = rs.uniform();
        const float xi_v = rs.uniform();
        const float xi_e = rs.uniform();
        const int j = cdf_search(P.cdf_pix, P.guide_pix, P.n_guide_pix, (double)xi_pix);
        const int iu = j % P.nu, iv = j / P.nu;
        const int eb = cdf_search(P.cdf_e, P.guide_e, P.n_guide_e, (double)xi_e);
        e = __ldg(P.bin_e + eb);
        if (REC) r_esrc = e;
        const float a_u = ((float)iu + xi_u - P.hu) * P.du;
        const float a_v = ((float)iv + xi_v - P.hv) * P.dv;
        const float t0 = J.f.P[0] + a_u * J.f.eu[0] + a_v * J.f.ev[0];
        const float t1 = J.f.P[1] + a_u * J.f.eu[1] + a_v * J.f.ev[1];
        const float t2 = J.f.P[2] + a_u * J.f.eu[2] + a_v * J.f.ev[2];
        dx = t0 - J.f.S[0];
        dy = t1 - J.f.S[1];
        dz = t2 - J.f.S[2];
        const float len = sqrtf(dx * dx + dy * dy + dz * dz);
        dx = dx / len;
        dy = dy / len;
        dz = dz / len;
        px = J.f.S[0]; py = J.f.S[1]; pz = J.f.S[2];

        // slab entry into the voxel box
        float tmin = 0.0f, tmax = (float)3.0e38;
        bool hit = true;
        const float d[3] = {dx, dy, dz};
        const float p[3] = {px, py, pz};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (d[a] != 0.0f) {
                float t1a = (P.lo[a] - p[a]) / d[a];
                float t2a = (P.hi[a] - p[a]) / d[a];
                if (t1a > t2a) { const float t = t1a; t1a = t2a; t2a = t; }
                if (t1a > tmin) tmin = t1a;
                if (t2a < tmax) tmax = t2a;
            } else if (p[a] < P.lo[a] || p[a] > P.hi[a]) {
                hit = false;
            }
        }
        if (tmin >= tmax) hit = false;
        if (!hit) {
            escape(P, k);
            return false;
        }
        px = px + tmin * dx;
        py = py + tmin * dy;
        pz = pz + tmin * dz;
        co.at(P, e);
        return true;
    }

    // One Woodcock free flight and what happens at its end; returns false
    // when the history is over.
    __device__ __forceinline__ bool step(const McParams& P, Counters& k) {
        if ((int)nsteps >= P.max_steps) {
            ++k.lim;
            record(P, OUT_STEP_LIMIT, -1, 0);
            return false;
        }
        const float xi_s = rs.uniform();
        const float s = -gd_logf(xi_s) / co.mumax;
        ++nsteps;
        ++k.steps;
        const float qx = px + s * dx, qy = py + s * dy, qz = pz + s * dz;
        const bool inside = (qx >= P.lo[0] && qx <= P.hi[0]) && (qy >= P.lo[1] && qy <= P.hi[1])
                         && (qz >= P.lo[2] && qz <= P.hi[2]);
        if (!inside) {
            move_to_box_exit(P);
            escape(P, k);
            return false;
        }
        px = qx; py = qy; pz = qz;

        // trilinear partial densities per material
        int i0[3], i1[3];
        float w0[3], w1[3];
        const float q[3] = {px, py, pz};
        const int dims[3] = {P.nx, P.ny, P.nz};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float fa = (q[a] - P.lo[a]) * P.ivox[a] - 0.5f;
            int f0 = (int)floorf(fa);
            const float t = fa - (float)f0;
            int f1 = f0 + 1;
            f0 = f0 < 0 ? 0 : (f0 > dims[a] - 1 ? dims[a] - 1 : f0);
            f1 = f1 < 0 ? 0 : (f1 > dims[a] - 1 ? dims[a] - 1 : f1);
            i0[a] = f0; i1[a] = f1;
            w0[a] = 1.0f - t; w1[a] = t;
        }
        float acc[NM];
#pragma unroll
        for (int m = 0; m < NM; ++m) acc[m] = 0.0f;
        const int sy = P.nx, sz = P.nx * P.ny;
#pragma unroll
        for (int corner = 0; corner < 8; ++corner) {
            const int cx = corner & 1, cy = (corner >> 1) & 1, cz = corner >> 2;
            const int v = (cx ? i1[0] : i0[0]) + sy * (cy ? i1[1] : i0[1]) + sz * (cz ? i1[2] : i0[2]);
            const float w = (cx ? w1[0] : w0[0]) * (cy ? w1[1] : w0[1]) * (cz ? w1[2] : w0[2]);
            const float a = w * __ldg(P.dens + v);
            const int mc = __ldg(P.mat + v);
#pragma unroll
            for (int m = 0; m < NM; ++m) acc[m] = acc[m] + (mc == m ? a : 0.0f);
        }
        float muR = 0.0f, muC = 0.0f, muP = 0.0f;
#pragma unroll
        for (int m = 0; m < NM; ++m) {
            muR = muR + acc[m] * co.r[m];
            muC = muC + acc[m] * co.c[m];
            muP = muP + acc[m] * co.p[m];
        }
        const float t = rs.uniform() * co.mumax;
        const float c1 = muR, c2 = c1 + muC, c3 = c2 + muP;
        if (t <= c1) {
            const float ct = rayleigh(rs);
            float cp, sp;
            azimuth(rs, cp, sp);
            rotate(dx, dy, dz, ct, cp, sp);
            scattered = 1;
            ++k.ray;
            if (REC) { ++r_ray; if (!r_first) r_first = 1; }
            return true;
        }
        if (t <= c2) {
            float ct, e2, cp, sp;
            compton(rs, e, ct, e2);
            azimuth(rs, cp, sp);
            rotate(dx, dy, dz, ct, cp, sp);
            scattered = 1;
            ++k.comp;
            if (REC) { ++r_comp; if (!r_first) r_first = 2; r_dep += (double)e - (double)e2; }
            e = e2;
            if (e < P.e_cut) {
                if (REC) r_dep += (double)e;
                ++k.cut;
                record(P, OUT_CUTOFF, -1, 0);
                return false;
            }
            co.at(P, e);
            return true;
        }
        if (t <= c3) {
            ++k.photo;
            if (REC) { if (!r_first) r_first = 3; r_dep += (double)e; }
            record(P, OUT_PHOTO, -1, 1);
            return false;
        }
        ++k.virt;
        if (REC) ++r_virt;
        return true;
    }
};

__device__ __forceinline__ void flush_counter(unsigned long long* dst, uint32_t v) {
    const uint32_t s = __reduce_add_sync(FULL, v);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(dst, (unsigned long long)s);
}

template <int NM, bool REC>
__global__ void __launch_bounds__(256) mc_kernel(const McParams P) {
    const int lane = threadIdx.x & 31;
    Lane<NM, REC> L;
    Counters k = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    bool alive = false;
    unsigned long long pool_next = 0, pool_end = 0;
    bool exhausted = false;
    int since_refill = P.refill_interval;

    for (;;) {
        if (!exhausted && (since_refill >= P.refill_interval || !__any_sync(FULL, alive))) {
            since_refill = 0;
            unsigned need = __ballot_sync(FULL, !alive);
            while (need) {
                if (pool_next >= pool_end) {
                    unsigned long long base = 0;
                    if (lane == 0) base = atomicAdd(P.counter, (unsigned long long)P.chunk);
                    base = __shfl_sync(FULL, base, 0);
                    if (base >= P.total) { exhausted = true; break; }
                    pool_next = base;
                    pool_end = base + (unsigned long long)P.chunk;
                    if (pool_end > P.total) pool_end = P.total;
                }
                const unsigned avail = (unsigned)(pool_end - pool_next);
                const unsigned want = (unsigned)__popc(need);
                const unsigned cnt = want < avail ? want : avail;
                const unsigned rank = (unsigned)__popc(need & ((1u << lane) - 1u));
                if (!alive && rank < cnt) alive = L.start(P, pool_next + rank, k);
                pool_next += cnt;
                need = __ballot_sync(FULL, !alive);
            }
        }
        ++since_refill;
        if (exhausted && !__any_sync(FULL, alive)) break;
        if (alive) alive = L.step(P, k);
    }

    flush_counter(P.stats + GDRR_ST_HISTORIES, k.hist);
    flush_counter(P.stats + GDRR_ST_STEPS, k.steps);
    flush_counter(P.stats + GDRR_ST_VIRTUAL, k.virt);
    flush_counter(P.stats + GDRR_ST_RAYLEIGH, k.ray);
    flush_counter(P.stats + GDRR_ST_COMPTON, k.comp);
    flush_counter(P.stats + GDRR_ST_PHOTO, k.photo);
    flush_counter(P.stats + GDRR_ST_TALLY_PRIMARY, k.tp);
    flush_counter(P.stats + GDRR_ST_TALLY_SCATTER, k.ts);
    flush_counter(P.stats + GDRR_ST_MISS, k.miss);
    flush_counter(P.stats + GDRR_ST_CUTOFF, k.cut);
    flush_counter(P.stats + GDRR_ST_STEP_LIMIT, k.lim);
}

__global__ void stream_words_kernel(uint64_t seed, uint32_t angle_index, uint64_t hid0, int n_hist,
                                    int n_blocks, uint32_t* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_hist) return;
    Stream rs;
    rs.init(seed, angle_index, hid0 + (uint64_t)i);
    uint32_t* o = out + (size_t)i * 4 * n_blocks;
    for (int w = 0; w < 4 * n_blocks; ++w) o[w] = rs.word();
}

template <int NM, bool REC>
cudaError_t launch_t(const McParams& p, int block, int grid, cudaStream_t s) {
    mc_kernel<NM, REC><<<grid, block, 0, s>>>(p);
    return cudaGetLastError();
}

template <int NM, bool REC>
int occupancy_t(int block) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, mc_kernel<NM, REC>, block, 0) != cudaSuccess) return 1;
    return n > 0 ? n : 1;
}

}  // namespace

cudaError_t launch_mc(const McParams& p, int block, int grid, bool records, cudaStream_t s) {
    if (records) {
        if (p.n_mat <= 2) return launch_t<2, true>(p, block, grid, s);
        if (p.n_mat <= 4) return launch_t<4, true>(p, block, grid, s);
        return launch_t<8, true>(p, block, grid, s);
    }
    if (p.n_mat <= 2) return launch_t<2, false>(p, block, grid, s);
    if (p.n_mat <= 4) return launch_t<4, false>(p, block, grid, s);
    return launch_t<8, false>(p, block, grid, s);
}

int mc_occupancy_blocks(int n_mat, int block, bool records) {
    if (records) {
        if (n_mat <= 2) return occupancy_t<2, true>(block);
        if (n_mat <= 4) return occupancy_t<4, true>(block);
        return occupancy_t<8, true>(block);
    }
    if (n_mat <= 2) return occupancy_t<2, false>(block);
    if (n_mat <= 4) return occupancy_t<4, false>(block);
    return occupancy_t<8, false>(block);
}

cudaError_t launch_stream_words(uint64_t seed, uint32_t angle_index, uint64_t hid0, int n_hist, int n_blocks,
                                uint32_t* out, cudaStream_t s) {
    if (n_hist <= 0) return cudaSuccess;
    stream_words_kernel<<<(n_hist + 127) / 128, 128, 0, s>>>(seed, angle_index, hid0, n_hist, n_blocks, out);
    return cudaGetLastError();
}

}  // namespace gdrr
