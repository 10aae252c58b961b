// Monte Carlo photon transport, Section 2.4 of the paper, for sm_103a.
//
// One CUDA thread tracks one photon history at a time (as in the paper), but
// the grid is persistent: warps claim chunks of histories from a global
// counter and refill lanes whose history ended, so lanes stay busy while
// histories of very different lengths finish.  The common event, a Woodcock
// free flight that ends in a virtual collision, runs every iteration; the
// rare, long branches (Rayleigh / Compton sampling, the detector tally, the
// start of a new history) are deferred: a lane that needs one waits, and once
// batch_min lanes of the warp wait, the warp serves them together.  Tallies
// are int64 fixed point (2^-24 keV), summed with integer atomics, so the
// result does not depend on which lane ran which history, when, or in which
// order.
//
// Data layout: one 8-byte record {density bits, material index} per voxel,
// in bricks of 4 x 2 x 2 voxels (one 128-byte cache line each), so each
// trilinear corner is a single 8-byte gather and the eight corners of a cell
// touch about 2.8 distinct lines instead of about 4.3 for a row-major layout;
// the per-lane energy-dependent coefficients live in shared memory, indexed
// by material, one column per thread.
//
// Most tentative collisions of Woodcock tracking are virtual (over 90 % in a
// torso, whose majorant is set by dense bone).  Before the eight corner
// gathers, a tentative collision is compared with a bound on mu over the
// macro cell that holds the corners (a small table: the largest density of
// each material per cell); above it the collision is virtual whatever the
// corners hold, and the gathers are skipped.  The bound never falls below the
// mu the gathers give, so every decision, draw and tally is the one plain
// Woodcock tracking makes.  A flight that passes the test waits, like the rare
// events, for the warp's service batch, where its gathers run together with
// those of the warp's other waiting lanes.
//
// Local majorants (an option, LM): the macro-cell bounds themselves serve as a
// piecewise-constant majorant.  A flight draws its optical depth tau = -ln xi
// and spends it cell by cell along the ray (a cell of bound b crossed whole
// costs b times its chord); where it runs out, tau / b into the cell, lies the
// tentative collision, real with probability mu / b (the same ordinate test,
// t = xi' b against the mixture).  Cheap cell crossings replace most of the
// flights (about 46 per history in the torso with the global majorant, 4 to 6
// with 16 to 32 mm cells); the tentative collisions wait for the service
// batch, where the gathers, the decision and the next flight's Philox block
// run on the warp's waiting lanes together.
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
//    counter = (block, angle index, history id lo, hi), one whole block per
//    draw site; uniforms are ((word >> 8) + 1) * 2^-24 in (0, 1];
//  * source: detector pixel from the fluence map w(u) and channel from the
//    spectrum phi(E), each by inverse CDF; uniform point inside the pixel;
//  * material at an off-centre point: trilinear mixture of the eight corner
//    voxels, mu_k(x, E) = sum_c w_c rho_c mu_hat_k(m_c, E) (the density
//    interpolation of Section 2.4, the same field the ray tracer of Section
//    2.3 integrates); the total decides real versus virtual, then one uniform
//    picks Rayleigh, Compton or photoelectric in that order;
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

// The macro-cell bound is raised by 2^-10, far above the rounding of the
// eight-corner mixture (eleven FP32 operations on the way to mu, each within
// 2^-24 relative), so mu as the kernel computes it never exceeds it.
constexpr float CELL_MARGIN = 1.0009765625f;

// Rejection samplers stop rejecting once their history has drawn this many
// Philox blocks and keep the candidate in hand (the azimuth takes phi = 0).
// A legal history stays far below it (at most max_steps flights plus a few
// tries per interaction, and every sampler accepts with probability at
// least 1/2); it bounds the loops for inputs that are not finite.
constexpr uint32_t MAX_BLOCKS = 1u << 24;

constexpr unsigned FULL = 0xffffffffu;

// Ten Philox rounds with the round keys k_r = key + r (0x9E3779B9, 0xBB67AE85)
// precomputed on the host (they depend only on the seed), so each round is
// two wide multiplies and two three-input XORs with a constant-bank operand.
// Each product is one 32 x 32 -> 64-bit multiply whose halves are the round's
// high and low words (0.6 % fewer instructions per flight than a low
// multiply beside a separate high multiply).
__device__ __forceinline__ void philox4x32_10(uint32_t& c0, uint32_t& c1, uint32_t& c2, uint32_t& c3,
                                              const RoundKeys& rk) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ rk.k0[r];
        const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ rk.k1[r];
        c0 = n0; c1 = (uint32_t)p1; c2 = n2; c3 = (uint32_t)p0;
    }
}

// The random stream of one history: Philox blocks with counter (k, angle
// index, history id lo, hi), k = 0, 1, 2, ...; every draw site takes the next
// whole block (source, each free flight, each rejection attempt), so the
// Philox rounds of a free flight run on all lanes of a warp together.
struct Stream {
    uint32_t angle, hlo, hhi, blk;

    __device__ __forceinline__ void init(uint32_t angle_index, uint64_t hid) {
        angle = angle_index; hlo = (uint32_t)hid; hhi = (uint32_t)(hid >> 32);
        blk = 0;
    }
    __device__ __forceinline__ uint4 block(const RoundKeys& rk) {
        uint32_t c0 = blk, c1 = angle, c2 = hlo, c3 = hhi;
        philox4x32_10(c0, c1, c2, c3, rk);
        ++blk;
        return make_uint4(c0, c1, c2, c3);
    }
};

// Uniform on (0, 1]: the top 24 bits plus one, times 2^-24 (exact in FP32).
__device__ __forceinline__ float uniform(uint32_t w) {
    return (float)((w >> 8) + 1u) * (float)(1.0 / 16777216.0);
}

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

// Inverse-CDF search in integers.  A uniform is xi = k 2^-24 with k the top
// 24 bits of its word plus one, and xi <= cdf[j] holds exactly when
// k <= floor(cdf[j] 2^24) = kcdf[j]; the smallest such j is the sample.  The
// guide table gives a start, two short scans finish.
__device__ __forceinline__ int cdf_search(const uint32_t* __restrict__ kcdf, const int* __restrict__ guide,
                                          int n_guide, uint32_t w) {
    const uint32_t k = (w >> 8) + 1u;
    int gi = (int)(((uint64_t)k * (uint64_t)n_guide) >> 24);
    gi = gi > n_guide - 1 ? n_guide - 1 : gi;
    int j = __ldg(guide + gi);
    while (j > 0 && k <= __ldg(kcdf + j - 1)) --j;
    while (k > __ldg(kcdf + j)) ++j;
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

__device__ __forceinline__ float response(const McParams& P, float e) {
    int ir; float f;
    interp_index(e, P.r0, P.inv_dr, P.n_r, ir, f);
    const float a = __ldg(P.resp + ir), b = __ldg(P.resp + ir + 1);
    return a + f * (b - a);
}

__device__ __forceinline__ void azimuth(Stream& rs, const RoundKeys& rk, float& cp, float& sp) {
    while (rs.blk < MAX_BLOCKS) {
        const uint4 w = rs.block(rk);
        const float a = 2.0f * uniform(w.x) - 1.0f;
        const float b = 2.0f * uniform(w.y) - 1.0f;
        const float r2 = a * a + b * b;
        if (r2 <= 1.0f && r2 > 0.0f) {
            const float inv = 1.0f / r2;
            cp = (a * a - b * b) * inv;
            sp = 2.0f * a * b * inv;
            return;
        }
    }
    cp = 1.0f;
    sp = 0.0f;
}

__device__ __forceinline__ void rotate(float& u, float& v, float& w, float ct, float cp, float sp) {
    const float st2 = 1.0f - ct * ct;
    const float st = st2 > 0.0f ? sqrtf(st2) : 0.0f;
    float nu_, nv_, nw_;
    if (w < (float)0.99999 && w > (float)-0.99999) {
        const float t = sqrtf(1.0f - w * w);
        const float sti = st / t;
        nu_ = u * ct + sti * (u * w * cp - v * sp);
        nv_ = v * ct + sti * (v * w * cp + u * sp);
        nw_ = w * ct - st * t * cp;
    } else {
        nu_ = st * cp;
        nv_ = st * sp;
        nw_ = w > 0.0f ? ct : -ct;
    }
    const float il = 1.0f / sqrtf(nu_ * nu_ + nv_ * nv_ + nw_ * nw_);
    u = nu_ * il;
    v = nv_ * il;
    w = nw_ * il;
}

// Rayleigh polar angle with the form factor of material m at energy e: the
// density of s = x^2 is F^2(s), linear in s between the table's nodes, so
// its cumulative is the trapezoid sum on the nodes and quadratic within an
// interval.  s is drawn on [0, s_max], s_max = (e / hc)^2, by inverse CDF
// (binary search for the interval, the root of the quadratic within it),
// cos = 1 - 2 s / s_max, and accepted with (1 + cos^2) / 2.  One block per
// attempt: word 0 draws s, word 1 the acceptance.
__device__ __forceinline__ float rayleigh_ff(Stream& rs, const McParams& P, float e, int m) {
    const float* __restrict__ S = P.ff_s;
    const float* __restrict__ A = P.ff_a + (size_t)m * P.n_ff;
    const float* __restrict__ G = P.ff_g + (size_t)m * P.n_ff;
    const float xmax = e * P.inv_hc;
    const float smax = xmax * xmax;
    int j = (int)(xmax * P.ff_idx);
    if (j > P.n_ff - 2) j = P.n_ff - 2;
    const float sj = __ldg(S + j), sj1 = __ldg(S + j + 1);
    const float gj = __ldg(G + j), gj1 = __ldg(G + j + 1);
    const float hj = sj1 - sj;
    const float tj = smax - sj;
    const float amax = __ldg(A + j) + tj * (gj + (gj1 - gj) * tj / (2.0f * hj));
    for (;;) {
        const uint4 w = rs.block(P.rk);
        const float target = uniform(w.x) * amax;
        int lo = 1, hi = j + 1;        // smallest k in [1, j+1] with A[k] >= target
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (__ldg(A + mid) >= target) hi = mid; else lo = mid + 1;
        }
        const float s0 = __ldg(S + lo - 1);
        const float h = __ldg(S + lo) - s0;
        const float g0 = __ldg(G + lo - 1), g1 = __ldg(G + lo);
        const float D = target - __ldg(A + lo - 1);
        float q = g0 * g0 + 2.0f * (g1 - g0) * D / h;
        if (q < 0.0f) q = 0.0f;
        float s = s0 + 2.0f * D / (g0 + sqrtf(q));
        if (s > smax) s = smax;
        float ct = 1.0f - 2.0f * s / smax;
        if (!(ct >= -1.0f)) ct = -1.0f;
        if (2.0f * uniform(w.y) <= 1.0f + ct * ct || rs.blk >= MAX_BLOCKS) return ct;
    }
}

// The polar angle of a Rayleigh or Compton event, in one rejection loop for
// both kinds: each attempt draws the history's next block and applies the
// event's own test, so a warp serving both kinds runs one Philox per attempt
// instead of one per kind.
//  * Rayleigh (Thomson law): mu = 2 a - 1 accepted when 2 b <= 1 + mu^2.
//  * Compton (Klein-Nishina, Kahn's method): with alpha = E / 511 keV, branch
//    r1 <= (1 + 2 alpha) / (9 + 2 alpha) takes x = 1 + 2 alpha r2 and accepts
//    when r3 <= 4 (x - 1) / x^2; else x = (1 + 2 alpha) / (1 + 2 alpha r2),
//    accepted when r3 <= (cos^2 + 1/x) / 2; cos = 1 - (x - 1) / alpha and
//    E' = E / x.
// A history that has drawn MAX_BLOCKS blocks keeps its candidate.
__device__ __forceinline__ void polar(Stream& rs, const RoundKeys& rk, bool ray, float e, float& ct_out,
                                      float& e_out) {
    const float alpha = e * (float)(1.0 / 510.99895);
    const float ialpha = (float)510.99895 / e;
    const float ta = 2.0f * alpha;
    float x = 1.0f, mu = 1.0f;
    for (;;) {
        const uint4 w = rs.block(rk);
        bool done;
        if (ray) {
            const float a = uniform(w.x);
            const float b = uniform(w.y);
            mu = 2.0f * a - 1.0f;
            done = 2.0f * b <= 1.0f + mu * mu || rs.blk >= MAX_BLOCKS;
        } else {
            const float r1 = uniform(w.x);
            const float r2 = uniform(w.y);
            const float r3 = uniform(w.z);
            if (r1 <= (1.0f + ta) / (9.0f + ta)) {
                x = 1.0f + ta * r2;
                done = r3 <= 4.0f * (x - 1.0f) / (x * x);
            } else {
                x = (1.0f + ta) / (1.0f + ta * r2);
                const float c = 1.0f - (x - 1.0f) * ialpha;
                done = r3 <= 0.5f * (c * c + 1.0f / x);
            }
            done = done || rs.blk >= MAX_BLOCKS;      // keep the last candidate
        }
        if (done) break;
    }
    if (ray) {
        ct_out = mu;
        e_out = e;
    } else {
        ct_out = 1.0f - (x - 1.0f) * ialpha;
        e_out = e / x;
    }
}

enum : uint32_t { OUT_PRIMARY = 0, OUT_SCATTER = 1, OUT_PHOTO = 2, OUT_CUTOFF = 3, OUT_MISS = 4, OUT_STEP_LIMIT = 5 };

// Lane states.  A lane whose history needs an interaction, a tally or a new
// history waits in one of the non-FLY states until enough lanes of its warp
// wait too; the warp then serves them together, which keeps the expensive
// rare branches from running with one or two active lanes.
enum : int { S_DEAD = 0, S_FLY = 1, S_RAY = 2, S_COMP = 3, S_ESC = 4, S_GATHER = 5 };

// What a local-majorant lane needs before it flies on (LM): a new flight
// (Philox block and optical depth), the reciprocal of a new direction, the
// cell of a new history's entry point.
enum : uint32_t { LM_DRAW = 1u, LM_DIR = 2u, LM_CELL = 4u, LM_ALL = 7u };

// Block-shared counters (GDRR_NSTATS), flushed to the stats array at exit.
__device__ __forceinline__ void count(unsigned long long* c, int k) { atomicAdd(c + k, 1ull); }

// GEN: the general kernel, which honours the nearest-voxel and scatter-filter
// options; the default kernel (GEN = false) carries neither.  LM: free flights
// with local majorants instead of the global one.
template <int NM, bool REC, bool GEN, bool LM = false>
struct Lane {
    float px, py, pz, dx, dy, dz, e;
    float mumax, inv_mumax;
    int state, scattered, job;
    uint32_t nsteps;
    uint32_t n_int;      // Compton interactions (low 16 bits) and Rayleigh (high 16 bits)
    int m_ray;           // material of the pending form-factor Rayleigh event (GEN)
    // thread totals of free flights, virtual collisions and cell-decided
    // virtual collisions.  Without GEN they are added once per history at its
    // end (flights = nsteps; cell-decided = flights that neither gathered nor
    // left the box), so the common free flight carries no counter updates.
    uint32_t c_steps, c_virt, c_skip;
    uint32_t ngath;      // flights of the current history that gathered corners (not GEN)
    bool defer_e;        // start / interact leave the energy tables to the caller
    bool need_e;         // ... which must then call set_energy(P, e) before the next flight
    float tg;            // t = xi mu_max of a flight waiting for its corner gathers
                         // (LM: xi until the flight's cell is known, then xi b)
    uint32_t wz;         // that flight block's third word (GEN: form-factor material pick)
    // LM: the flight's remaining optical depth, the direction's reciprocals,
    // the cell of the position, what the lane needs next (LM_*) and the
    // thread's count of cell crossings
    float tau, idx, idy, idz;
    int cx, cy, cz;
    uint32_t lm_need, c_cross;
    Stream rs;
    // per-thread coefficient tables in shared memory: coef[k][m][tid],
    // k = 0 total, 1 Rayleigh, 2 Compton (photoelectric is the remainder)
    float* coef;
    int stride;          // blockDim.x
    // event record (REC only)
    uint64_t gidx;
    uint32_t r_virt, r_ray, r_comp, r_first, r_raymat;
    float r_esrc;
    double r_dep;

    __device__ __forceinline__ float& cf(int k, int m) { return coef[(k * NM + m) * stride]; }

    // Largest total mu at the lane's energy over a macro cell's voxels: the
    // cell's per-material maximum densities times the lane's coefficients.
    // Every corner's term rho_c mu_m(E) is at most this, and the trilinear
    // weights sum to one, so the mixture mu is at most it too.
    __device__ __forceinline__ float cell_bound(const McParams& P, int cell) {
        const float* r = P.cells + (size_t)cell * NM;
        float b;
        if constexpr (NM == 2) {
            const float2 v = __ldg(reinterpret_cast<const float2*>(r));
            b = fmaxf(v.x * cf(0, 0), v.y * cf(0, 1));
        } else {
            b = 0.0f;
#pragma unroll
            for (int q = 0; q < NM; q += 4) {
                const float4 v = __ldg(reinterpret_cast<const float4*>(r + q));
                b = fmaxf(b, fmaxf(fmaxf(v.x * cf(0, q), v.y * cf(0, q + 1)),
                                   fmaxf(v.z * cf(0, q + 2), v.w * cf(0, q + 3))));
            }
        }
        return b * CELL_MARGIN;
    }

    __device__ __forceinline__ void set_energy(const McParams& P, float en) {
        e = en;
        int ie; float f;
        interp_index(en, P.e0, P.inv_de, P.n_e, ie, f);
#pragma unroll
        for (int m = 0; m < NM; ++m) {
            float r = 0.0f, c = 0.0f, t = 0.0f;
            if (m < P.n_mat) {
                const float* tb = P.tab + (size_t)m * 3 * P.n_e;
                const float r0 = __ldg(tb + ie), r1 = __ldg(tb + ie + 1);
                const float c0 = __ldg(tb + P.n_e + ie), c1 = __ldg(tb + P.n_e + ie + 1);
                const float p0 = __ldg(tb + 2 * P.n_e + ie), p1 = __ldg(tb + 2 * P.n_e + ie + 1);
                r = r0 + f * (r1 - r0);
                c = c0 + f * (c1 - c0);
                const float p = p0 + f * (p1 - p0);
                t = (r + c) + p;
            }
            cf(0, m) = t;
            cf(1, m) = r;
            cf(2, m) = c;
        }
        const float a = __ldg(P.major + ie), b = __ldg(P.major + ie + 1);
        mumax = a > b ? a : b;
        inv_mumax = 1.0f / mumax;
    }

    // a history ended; esc: its last flight left the box
    __device__ __forceinline__ void end_counts(uint32_t esc) {
        if (GEN) return;
        if (LM) {                    // no cell test: every virtual collision gathered
            c_steps += nsteps;
            return;
        }
        const uint32_t skipped = nsteps - ngath - esc;
        c_steps += nsteps;
        c_skip += skipped;
        c_virt += skipped;
    }

    __device__ __forceinline__ void record(const McParams& P, uint32_t outcome, int pixel, uint32_t photo) {
        if (!REC) return;
        gdrr_history_record r;
        r.n_steps = nsteps; r.n_virtual = r_virt; r.n_rayleigh = r_ray; r.n_compton = r_comp;
        r.n_photo = photo; r.outcome = outcome; r.rng_blocks = rs.blk; r.first_interaction = r_first;
        r.pixel = pixel; r.e_source = r_esrc; r.e_final = e; r.ray_material = r_raymat; r.e_deposited = r_dep;
        P.records[gidx] = r;
    }

    // Straight line from the box surface (or the source) to the imager
    // plane; tally r(E) at the pixel it meets (Section 2.4).  A lane that
    // left the box in a free flight first moves from its last position inside
    // to the box surface along its direction.
    __device__ __forceinline__ void escape(const McParams& P, unsigned long long* cnt, bool from_inside) {
        if (from_inside) move_to_box_exit(P);
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
                bool take = true;            // scatter filter (Section 2.4)
                if (GEN && scattered && P.scatter_filter) {
                    const uint32_t nc = n_int & 0xffffu, nr = n_int >> 16;
                    take = P.scatter_filter == 1 ? (nc == 1 && nr == 0)
                         : (P.scatter_filter == 2 ? (nr == 1 && nc == 0) : (nc + nr >= 2));
                }
                if (take && fu >= 0.0f && fu < (float)P.nu && fv >= 0.0f && fv < (float)P.nv) {
                    pixel = (int)fv * P.nu + (int)fu;
                    const long long q = llrintf(response(P, e) * 16777216.0f);
                    int64_t* t = scattered ? J.tally_s : J.tally_p;
                    atomicAdd(reinterpret_cast<unsigned long long*>(t + pixel), (unsigned long long)q);
                    outcome = scattered ? OUT_SCATTER : OUT_PRIMARY;
                }
            }
        }
        count(cnt, outcome == OUT_PRIMARY ? GDRR_ST_TALLY_PRIMARY
                                          : (outcome == OUT_SCATTER ? GDRR_ST_TALLY_SCATTER : GDRR_ST_MISS));
        record(P, outcome, pixel, 0);
        end_counts(from_inside ? 1u : 0u);
        state = S_DEAD;
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

    // Start flattened history g: source sampling and box entry.  Leaves the
    // lane FLY, or DEAD after tallying a photon that misses the box.
    __device__ __forceinline__ void start(const McParams& P, uint64_t g, unsigned long long* cnt) {
        gidx = g;
        int lo = 0, hi = P.n_jobs - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (P.jobs[mid].first <= g) lo = mid; else hi = mid - 1;
        }
        job = lo;
        const Job& J = P.jobs[job];
        const uint64_t hid = J.hid_offset + (g - J.first);
        rs.init(J.angle_index, hid);
        count(cnt, GDRR_ST_HISTORIES);
        nsteps = 0;
        ngath = 0;
        scattered = 0;
        if (GEN) n_int = 0;
        if (REC) { r_virt = 0; r_ray = 0; r_comp = 0; r_first = 0; r_raymat = 0; r_dep = 0.0; }

        const uint4 w0 = rs.block(P.rk);
        const float xi_u = uniform(w0.y);
        const float xi_v = uniform(w0.z);
        const int j = cdf_search(P.kcdf_pix, P.guide_pix, P.n_guide_pix, w0.x);
        const int iu = j % P.nu, iv = j / P.nu;
        const int ecol = P.e_col ? iu : 0;   // per-column spectrum row (energy-dependent bowtie)
        const int eb = cdf_search(P.kcdf_e + ecol * P.n_bins, P.guide_e + ecol * P.n_guide_e, P.n_guide_e, w0.w);
        const float en = __ldg(P.bin_e + eb);
        if (REC) r_esrc = en;
        const float a_u = ((float)iu + xi_u - P.hu) * P.du;
        const float a_v = ((float)iv + xi_v - P.hv) * P.dv;
        const float t0 = J.f.P[0] + a_u * J.f.eu[0] + a_v * J.f.ev[0];
        const float t1 = J.f.P[1] + a_u * J.f.eu[1] + a_v * J.f.ev[1];
        const float t2 = J.f.P[2] + a_u * J.f.eu[2] + a_v * J.f.ev[2];
        dx = t0 - J.f.S[0];
        dy = t1 - J.f.S[1];
        dz = t2 - J.f.S[2];
        const float il = 1.0f / sqrtf(dx * dx + dy * dy + dz * dz);
        dx = dx * il;
        dy = dy * il;
        dz = dz * il;
        px = J.f.S[0]; py = J.f.S[1]; pz = J.f.S[2];
        e = en;

        float tmin = 0.0f, tmax = (float)3.0e38;
        bool hit = true;
        const float d[3] = {dx, dy, dz};
        const float p[3] = {px, py, pz};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (d[a] != 0.0f) {
                const float id = 1.0f / d[a];
                float t1a = (P.lo[a] - p[a]) * id;
                float t2a = (P.hi[a] - p[a]) * id;
                if (t1a > t2a) { const float t = t1a; t1a = t2a; t2a = t; }
                if (t1a > tmin) tmin = t1a;
                if (t2a < tmax) tmax = t2a;
            } else if (p[a] < P.lo[a] || p[a] > P.hi[a]) {
                hit = false;
            }
        }
        if (tmin >= tmax) hit = false;
        if (!hit) {
            escape(P, cnt, false);
            return;
        }
        px = px + tmin * dx;
        py = py + tmin * dy;
        pz = pz + tmin * dz;
        if (defer_e) need_e = true; else set_energy(P, en);
        if (LM) lm_need = LM_ALL;
        state = S_FLY;
    }

    // Start history P.seg0 + i from the source pass's record: the state
    // start() leaves (source block drawn, position at the box entry, energy
    // tables pending), or nothing when the history already ended there.
    __device__ __forceinline__ void start_src(const McParams& P, uint64_t i) {
        const float4 b = __ldcs(P.src + 2 * i + 1);
        const uint32_t j1 = __float_as_uint(b.w);
        if (j1 == 0u) return;
        const float4 a = __ldcs(P.src + 2 * i);
        const uint64_t g = P.seg0 + i;
        gidx = g;
        job = (int)j1 - 1;
        const Job& J = P.jobs[job];
        rs.init(J.angle_index, J.hid_offset + (g - J.first));
        rs.blk = 1;
        nsteps = 0;
        ngath = 0;
        scattered = 0;
        px = a.x; py = a.y; pz = a.z;
        dx = a.w; dy = b.x; dz = b.y;
        e = b.z;
        if (defer_e) need_e = true; else set_energy(P, e);
        if (LM) lm_need = LM_ALL;
        state = S_FLY;
    }

    // One Woodcock free flight and the real/virtual decision at its end.
    __device__ __forceinline__ void step(const McParams& P, unsigned long long* cnt) {
        if ((int)nsteps >= P.max_steps) {
            count(cnt, GDRR_ST_STEP_LIMIT);
            record(P, OUT_STEP_LIMIT, -1, 0);
            end_counts(0u);
            state = S_DEAD;
            return;
        }
        const uint4 wf = rs.block(P.rk);            // this flight's block
        const float s = -gd_logf(uniform(wf.x)) * inv_mumax;
        ++nsteps;
        if (GEN) ++c_steps;
        const float qx = px + s * dx, qy = py + s * dy, qz = pz + s * dz;
        const bool inside = (qx >= P.lo[0] && qx <= P.hi[0]) && (qy >= P.lo[1] && qy <= P.hi[1])
                         && (qz >= P.lo[2] && qz <= P.hi[2]);
        if (!inside) {
            state = S_ESC;           // the box exit and tally wait for the warp's batch
            return;
        }
        px = qx; py = qy; pz = qz;

        if (GEN && P.nearest_voxel) {
            // no density interpolation: the voxel containing the point
            const int gx = min(max((int)floorf((px - P.lo[0]) * P.ivox[0]), 0), P.nx - 1);
            const int gy = min(max((int)floorf((py - P.lo[1]) * P.ivox[1]), 0), P.ny - 1);
            const int gz = min(max((int)floorf((pz - P.lo[2]) * P.ivox[2]), 0), P.nz - 1);
            const uint2 vx = __ldg(P.vox + brick_x(gx) + brick_y(gy, P.bsy) + brick_z(gz, P.bsz));
            const float a0 = __uint_as_float(vx.x);
            const int m0 = (int)vx.y;
            const float t = uniform(wf.y) * mumax;
            if (t > a0 * cf(0, m0)) {
                ++c_virt;
                if (REC) ++r_virt;
                return;
            }
            const float muR = a0 * cf(1, m0), muC = a0 * cf(2, m0);
            m_ray = m0;
            real_collision(P, t, muR, muC, cnt);
            return;
        }

        // the lower trilinear corner, computed as gather() computes it,
        // locates the macro cell
        const int x0 = max((int)floorf((px - P.lo[0]) * P.ivox[0] - 0.5f), 0);
        const int y0 = max((int)floorf((py - P.lo[1]) * P.ivox[1] - 0.5f), 0);
        const int z0 = max((int)floorf((pz - P.lo[2]) * P.ivox[2] - 0.5f), 0);
        const float t = uniform(wf.y) * mumax;
        if (P.cells) {
            // the corners lie in [x0, x0 + 1] etc., inside the cover of x0's cell:
            // above the cell's bound the collision is virtual whatever they hold
            const int cell = (x0 >> P.cshift) + P.ncx * ((y0 >> P.cshift) + P.ncy * (z0 >> P.cshift));
            if (t > cell_bound(P, cell)) {
                if (GEN) { ++c_virt; ++c_skip; }
                if (REC) ++r_virt;
                return;
            }
        }
        // the corner gathers wait for the warp's service batch
        tg = t;
        if (GEN) wz = wf.z;
        state = S_GATHER;
    }

    // The boundary plane between cells j - 1 and j of axis a (n cells): the
    // box faces for j = 0 and j = n, else where the lower trilinear corner
    // index reaches j 2^s, i.e. (x - lo) / vox - 1/2 = j 2^s.
    __device__ __forceinline__ static float lm_plane(const McParams& P, int a, int j, int n) {
        if (j <= 0) return P.lo[a];
        if (j >= n) return P.hi[a];
        return P.lo[a] + ((float)(j << P.cshift) + 0.5f) * P.vox_mm[a];
    }

    // LM, in the service batch: the entry cell of a new history, the
    // reciprocals of a new direction, and the next flight: its Philox block,
    // its optical depth tau = -ln xi and the uniform of its ordinate test.
    __device__ __forceinline__ void lm_prepare(const McParams& P, unsigned long long* cnt) {
        if (lm_need & LM_CELL) {
            const int gx = max((int)floorf((px - P.lo[0]) * P.ivox[0] - 0.5f), 0) >> P.cshift;
            const int gy = max((int)floorf((py - P.lo[1]) * P.ivox[1] - 0.5f), 0) >> P.cshift;
            const int gz = max((int)floorf((pz - P.lo[2]) * P.ivox[2] - 0.5f), 0) >> P.cshift;
            cx = min(gx, P.ncx - 1);
            cy = min(gy, P.ncy - 1);
            cz = min(gz, P.ncz - 1);
        }
        if (lm_need & LM_DIR) {
            idx = dx != 0.0f ? 1.0f / dx : 0.0f;
            idy = dy != 0.0f ? 1.0f / dy : 0.0f;
            idz = dz != 0.0f ? 1.0f / dz : 0.0f;
        }
        lm_need = 0u;
        if ((int)nsteps >= P.max_steps) {
            count(cnt, GDRR_ST_STEP_LIMIT);
            record(P, OUT_STEP_LIMIT, -1, 0);
            end_counts(0u);
            state = S_DEAD;
            return;
        }
        const uint4 wf = rs.block(P.rk);
        ++nsteps;
        if (GEN) ++c_steps;
        tau = -gd_logf(uniform(wf.x));
        tg = uniform(wf.y);
        if (GEN) wz = wf.z;
    }

    // LM: one cell of a flight.  With b the cell's bound and tx the distance
    // to its exit, the remaining depth either runs out inside (the tentative
    // collision lies tau / b ahead and waits for the warp's service batch) or
    // pays b tx, and the lane moves to the exit point and on to the next cell
    // (one step along every axis whose exit plane is nearest, all of them on
    // a tie).  Every crossing moves the cell along the direction of flight, so
    // a flight crosses at most ncx + ncy + ncz cells; leaving the grid leaves
    // the box, from the last position inside.
    __device__ __forceinline__ void walk(const McParams& P) {
        const float b = cell_bound(P, cx + P.ncx * (cy + P.ncy * cz));
        float tx = (float)3.0e38, ty = tx, tz = tx;
        if (dx > 0.0f) tx = (lm_plane(P, 0, cx + 1, P.ncx) - px) * idx;
        else if (dx < 0.0f) tx = (lm_plane(P, 0, cx, P.ncx) - px) * idx;
        if (dy > 0.0f) ty = (lm_plane(P, 1, cy + 1, P.ncy) - py) * idy;
        else if (dy < 0.0f) ty = (lm_plane(P, 1, cy, P.ncy) - py) * idy;
        if (dz > 0.0f) tz = (lm_plane(P, 2, cz + 1, P.ncz) - pz) * idz;
        else if (dz < 0.0f) tz = (lm_plane(P, 2, cz, P.ncz) - pz) * idz;
        if (dx != 0.0f && !(tx > 0.0f)) tx = 0.0f;       // already on the plane
        if (dy != 0.0f && !(ty > 0.0f)) ty = 0.0f;
        if (dz != 0.0f && !(tz > 0.0f)) tz = 0.0f;
        const float t = fminf(tx, fminf(ty, tz));
        const float bt = b * t;
        if (tau < bt) {
            const float s = tau / b;
            px = px + s * dx;
            py = py + s * dy;
            pz = pz + s * dz;
            tg = tg * b;
            state = S_GATHER;
            return;
        }
        tau = tau - bt;
        const bool sx = dx != 0.0f && tx == t, sy = dy != 0.0f && ty == t, sz = dz != 0.0f && tz == t;
        const int nx_ = sx ? cx + (dx > 0.0f ? 1 : -1) : cx;
        const int ny_ = sy ? cy + (dy > 0.0f ? 1 : -1) : cy;
        const int nz_ = sz ? cz + (dz > 0.0f ? 1 : -1) : cz;
        if (!(sx || sy || sz) || nx_ < 0 || nx_ >= P.ncx || ny_ < 0 || ny_ >= P.ncy || nz_ < 0 || nz_ >= P.ncz) {
            state = S_ESC;
            return;
        }
        px = px + t * dx;
        py = py + t * dy;
        pz = pz + t * dz;
        cx = nx_; cy = ny_; cz = nz_;
        ++c_cross;
    }

    // The deferred part of a free flight that passed the macro-cell test:
    // the eight-corner mixture at the lane's position and the real/virtual
    // decision for its t.  The warp serves its waiting lanes together, so the
    // gathers run on many lanes at once instead of on the few whose flights
    // passed the test in one iteration.
    __device__ __forceinline__ void gather(const McParams& P, unsigned long long* cnt) {
        if (!GEN) ++ngath;
        const float t = tg;
        if (LM && GEN && P.nearest_voxel) {
            // no density interpolation: the voxel containing the point
            const int gx = min(max((int)floorf((px - P.lo[0]) * P.ivox[0]), 0), P.nx - 1);
            const int gy = min(max((int)floorf((py - P.lo[1]) * P.ivox[1]), 0), P.ny - 1);
            const int gz = min(max((int)floorf((pz - P.lo[2]) * P.ivox[2]), 0), P.nz - 1);
            const uint2 vx = __ldg(P.vox + brick_x(gx) + brick_y(gy, P.bsy) + brick_z(gz, P.bsz));
            const float a0 = __uint_as_float(vx.x);
            const int m0 = (int)vx.y;
            if (t > a0 * cf(0, m0)) {
                ++c_virt;
                if (REC) ++r_virt;
                lm_need |= LM_DRAW;
                state = S_FLY;
                return;
            }
            m_ray = m0;
            real_collision(P, t, a0 * cf(1, m0), a0 * cf(2, m0), cnt);
            return;
        }
        const float fx = (px - P.lo[0]) * P.ivox[0] - 0.5f;
        const float fy = (py - P.lo[1]) * P.ivox[1] - 0.5f;
        const float fz = (pz - P.lo[2]) * P.ivox[2] - 0.5f;
        const int gx = (int)floorf(fx), gy = (int)floorf(fy), gz = (int)floorf(fz);
        const float tx = fx - (float)gx, ty = fy - (float)gy, tz = fz - (float)gz;
        // inside the box f lies in [-1/2, n - 1/2], so g in [-1, n - 1]: the
        // lower corner clamps only from below, the upper only from above
        const int x0 = max(gx, 0), x1 = min(gx + 1, P.nx - 1);
        const int y0 = max(gy, 0), y1 = min(gy + 1, P.ny - 1);
        const int z0 = max(gz, 0), z1 = min(gz + 1, P.nz - 1);
        const float wx0 = 1.0f - tx, wy0 = 1.0f - ty, wz0 = 1.0f - tz;
        const float wxy[4] = {wx0 * wy0, tx * wy0, wx0 * ty, tx * ty};
        const int bx[2] = {brick_x(x0), brick_x(x1)};
        const int by[2] = {brick_y(y0, P.bsy), brick_y(y1, P.bsy)};
        const int bz[2] = {brick_z(z0, P.bsz), brick_z(z1, P.bsz)};
        const int rows[4] = {by[0] + bz[0], by[1] + bz[0], by[0] + bz[1], by[1] + bz[1]};
        float a[8];
        int mc[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int v = rows[c >> 1] + bx[c & 1];
            const uint2 vx = __ldg(P.vox + v);
            a[c] = (wxy[c & 3] * ((c >> 2) ? tz : wz0)) * __uint_as_float(vx.x);
            mc[c] = (int)vx.y;
        }
        float muT = a[0] * cf(0, mc[0]);
#pragma unroll
        for (int c = 1; c < 8; ++c) muT = muT + a[c] * cf(0, mc[c]);
        if (t > muT) {
            ++c_virt;
            if (REC) ++r_virt;
            if (LM) lm_need |= LM_DRAW;
            state = S_FLY;
            return;
        }
        float muR = a[0] * cf(1, mc[0]);
#pragma unroll
        for (int c = 1; c < 8; ++c) muR = muR + a[c] * cf(1, mc[c]);
        float muC = a[0] * cf(2, mc[0]);
#pragma unroll
        for (int c = 1; c < 8; ++c) muC = muC + a[c] * cf(2, mc[c]);
        if (GEN && P.ray_ff && t <= muR) {
            // the form factor's material: the corner whose Rayleigh share of
            // mu_R holds xi mu_R, xi the flight block's third word
            const float target = uniform(wz) * muR;
            float acc = 0.0f;
            m_ray = mc[7];
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                acc = acc + a[c] * cf(1, mc[c]);
                if (target <= acc) { m_ray = mc[c]; break; }
            }
        }
        real_collision(P, t, muR, muC, cnt);
    }

    // A real collision: Rayleigh if t <= mu_R, Compton if t <= mu_R + mu_C,
    // else photoelectric absorption.
    __device__ __forceinline__ void real_collision(const McParams& P, float t, float muR, float muC,
                                                   unsigned long long* cnt) {
        if (t <= muR) {
            state = S_RAY;
        } else if (t <= muR + muC) {
            state = S_COMP;
        } else {
            count(cnt, GDRR_ST_PHOTO);
            if (REC) { if (!r_first) r_first = 3; r_dep += (double)e; }
            record(P, OUT_PHOTO, -1, 1);
            end_counts(0u);
            state = S_DEAD;
        }
    }

    // The deferred Rayleigh or Compton interaction of a waiting lane.  The
    // polar angle comes from the event's own sampler; the azimuth and the
    // rotation are common code, so a batch holding both kinds runs them once.
    __device__ __forceinline__ void interact(const McParams& P, unsigned long long* cnt) {
        const bool ray = state == S_RAY;
        float ct, e2 = e;
        if (GEN && ray && P.ray_ff) {
            ct = rayleigh_ff(rs, P, e, m_ray);
            if (REC) r_raymat = (uint32_t)m_ray;
        } else {
            polar(rs, P.rk, ray, e, ct, e2);
        }
        float cp, sp;
        azimuth(rs, P.rk, cp, sp);
        rotate(dx, dy, dz, ct, cp, sp);
        scattered = 1;
        if (ray) {
            if (GEN) n_int += 0x10000u;
            count(cnt, GDRR_ST_RAYLEIGH);
            if (REC) { ++r_ray; if (!r_first) r_first = 1; }
            if (LM) lm_need |= LM_DRAW | LM_DIR;
            state = S_FLY;
            return;
        }
        if (GEN) n_int += 1u;
        count(cnt, GDRR_ST_COMPTON);
        if (REC) { ++r_comp; if (!r_first) r_first = 2; r_dep += (double)e - (double)e2; }
        if (e2 < P.e_cut) {
            e = e2;
            if (REC) r_dep += (double)e;
            count(cnt, GDRR_ST_CUTOFF);
            record(P, OUT_CUTOFF, -1, 0);
            end_counts(0u);
            state = S_DEAD;
            return;
        }
        if (defer_e) {
            e = e2;
            need_e = true;
        } else {
            set_energy(P, e2);
        }
        if (LM) lm_need |= LM_DRAW | LM_DIR;
        state = S_FLY;
    }
};

template <int NM, bool REC, bool GEN, bool LM>
// Up to 512 threads per block, 64 registers per thread (the same cap at 2 x 512
// or 4 x 256 resident threads): the autotuner's block sizes 64 ... 512.
__global__ void __launch_bounds__(512, 2) mc_kernel(const McParams P) {
    extern __shared__ float smem[];
    __shared__ unsigned long long cnt[GDRR_NSTATS];
    for (int i = threadIdx.x; i < GDRR_NSTATS; i += blockDim.x) cnt[i] = 0ull;
    __syncthreads();

    const int lane = threadIdx.x & 31;
    Lane<NM, REC, GEN, LM> L;
    L.coef = smem + threadIdx.x;
    L.stride = blockDim.x;
    L.state = S_DEAD;
    L.defer_e = true;                 // new histories and Compton events share one table pass
    L.need_e = false;
    L.c_steps = 0; L.c_virt = 0; L.c_skip = 0;
    L.lm_need = 0u; L.c_cross = 0u;
    unsigned long long pool_next = 0, pool_end = 0;
    bool exhausted = false;

    for (;;) {
        const unsigned fly = __ballot_sync(FULL, L.state == S_FLY);
        if (32 - __popc(fly) >= P.batch_min || fly == 0u) {
            // serve waiting lanes together: corner gathers, interactions,
            // tallies, new histories
            if (L.state == S_GATHER) L.gather(P, cnt);
            if (L.state == S_RAY || L.state == S_COMP) L.interact(P, cnt);
            if (L.state == S_ESC) L.escape(P, cnt, true);
            if (!exhausted) {
                unsigned need = __ballot_sync(FULL, L.state == S_DEAD);
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
                    const unsigned take = want < avail ? want : avail;
                    const unsigned rank = (unsigned)__popc(need & ((1u << lane) - 1u));
                    if (((need >> lane) & 1u) && rank < take) {
                        if (!REC && !GEN && P.src) L.start_src(P, pool_next + rank);
                        else L.start(P, P.seg0 + pool_next + rank, cnt);
                    }
                    pool_next += take;
                    need = __ballot_sync(FULL, L.state == S_DEAD);
                }
            }
            if (L.need_e) {
                L.set_energy(P, L.e);
                L.need_e = false;
            }
            if (LM && L.lm_need) L.lm_prepare(P, cnt);
            if (exhausted && !__any_sync(FULL, L.state != S_DEAD)) break;
        }
        if (L.state == S_FLY) {
            if constexpr (LM) L.walk(P);
            else L.step(P, cnt);
        }
    }

    atomicAdd(&cnt[GDRR_ST_STEPS], (unsigned long long)L.c_steps);
    atomicAdd(&cnt[GDRR_ST_VIRTUAL], (unsigned long long)L.c_virt);
    atomicAdd(&cnt[GDRR_ST_CELL_SKIPS], (unsigned long long)L.c_skip);
    if (LM) atomicAdd(&cnt[GDRR_ST_CELL_CROSSINGS], (unsigned long long)L.c_cross);
    __syncthreads();
    for (int i = threadIdx.x; i < GDRR_NSTATS; i += blockDim.x)
        if (cnt[i]) atomicAdd(P.stats + i, cnt[i]);
}

// ---------------------------------------------------------------------------
// The source pass: Lane::start for every history of the launch, on full
// warps (one history per thread), apart from the transport's service
// batches.  A history that misses the box is tallied and counted here; the
// others leave their state (position at the box entry, direction, energy)
// for Lane::start_src.  The arithmetic is start()'s, call for call, so the
// transport's draws, decisions and tallies do not change.
template <int NM>
__global__ void __launch_bounds__(256) mc_source_kernel(const McParams P, float4* __restrict__ out) {
    __shared__ unsigned long long cnt[GDRR_NSTATS];
    for (int i = threadIdx.x; i < GDRR_NSTATS; i += blockDim.x) cnt[i] = 0ull;
    __syncthreads();
    Lane<NM, false, false> L;
    L.coef = nullptr;
    L.stride = 0;
    L.defer_e = true;
    L.need_e = false;
    L.c_steps = 0; L.c_virt = 0; L.c_skip = 0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P.total;
         i += (uint64_t)gridDim.x * blockDim.x) {
        L.state = S_DEAD;
        L.start(P, P.seg0 + i, cnt);
        float4 a = make_float4(0.0f, 0.0f, 0.0f, 0.0f), b = a;
        if (L.state == S_FLY) {
            a = make_float4(L.px, L.py, L.pz, L.dx);
            b = make_float4(L.dy, L.dz, L.e, __uint_as_float((uint32_t)L.job + 1u));
        }
        __stcs(out + 2 * i, a);
        __stcs(out + 2 * i + 1, b);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < GDRR_NSTATS; i += blockDim.x)
        if (cnt[i]) atomicAdd(P.stats + i, cnt[i]);
}

// ---------------------------------------------------------------------------
// The photon-pool form of the same transport.
//
// In mc_kernel a lane keeps its photon from birth to death, so a warp flies
// only the lanes that are not waiting for a service, and serves its waiting
// lanes on partial warps.  Here a block of 8 warps shares a pool of photons
// in shared memory and moves them between warps: every phase runs the
// photons that need it on full warps.  A round of the block is
//   START   free slots take new histories (source sampling, box entry);
//   FLIGHT  each lane flies a photon until its flight needs the corner
//           gathers or leaves the box, parks it, and takes the next ready
//           photon of its class;
//   GATHER  the eight-corner mixture of the parked flights: virtual, real;
//   INTER   Rayleigh / Compton sampling of the real collisions;
//   ESCAPE  box exit and imager tally;
// with a block barrier between phases.  Lane l of every warp serves pool
// class l only: class l holds K slots, and field f of slot s sits at word
// (f K + s) 32 + l, so a warp's 32 lanes touch 32 different banks whatever
// slots they hold.  Each class keeps queues of slot numbers per phase; a
// queue's entry j goes to warp j mod 8, which packs the work into full warps.
// The arithmetic per photon is Lane's, call for call (start, step, gather,
// interact, escape), so every history's draws, decisions and tally are the
// ones mc_kernel and the oracle produce; only the order in which histories
// advance differs, and the integer tallies and counters do not depend on it.
enum : int {
    PF_PX, PF_PY, PF_PZ, PF_DX, PF_DY, PF_DZ, PF_E, PF_MUMAX, PF_INVMU, PF_TG,
    PF_STATE, PF_JOB, PF_NSTEPS, PF_NGATH, PF_ANGLE, PF_HLO, PF_HHI, PF_BLK, PF_N
};
// queues (slot numbers, one byte each): ready by round parity, gather,
// interaction, escape, free by round parity
enum : int { PQ_R0, PQ_R1, PQ_G, PQ_I, PQ_E, PQ_F0, PQ_F1, PQ_N };
// per-class counters: queue lengths (by queue), the ready queue's read head
enum : int { PC_HEAD = PQ_N, PC_N };

// A block barrier reached by a converged warp.  The phases end in per-lane
// loops of different lengths, and an aligned barrier (bar.sync) that a warp
// reaches in several diverged groups can release before another warp has
// arrived; reconverging the warp first keeps every phase's queue updates
// ahead of the next phase.
__device__ __forceinline__ void block_sync() {
    __syncwarp();
    __syncthreads();
}

constexpr int POOL_WARPS = 8;
constexpr int POOL_THREADS = 32 * POOL_WARPS;

// Queue entries are whole 32-bit words: entries of different classes written
// by different warps at the same time never share a word.
template <int NM>
constexpr size_t pool_smem_bytes(int K) {
    return (size_t)(PF_N + 3 * NM) * K * 32 * sizeof(float) + (size_t)PQ_N * K * 32 * sizeof(int) +
           (size_t)PC_N * 32 * sizeof(int);
}

template <int NM>
struct Pool {
    uint32_t* fld;     // [PF_N][K][32]
    float* cf;         // [3 NM][K][32]
    int* q;            // [PQ_N][K][32] slot numbers
    int* n;            // [PC_N][32]
    int K;

    __device__ __forceinline__ uint32_t& u(int f, int s, int l) { return fld[(f * K + s) * 32 + l]; }
    __device__ __forceinline__ float& fl(int f, int s, int l) { return reinterpret_cast<float*>(fld)[(f * K + s) * 32 + l]; }
    __device__ __forceinline__ int& slot(int queue, int j, int l) { return q[(queue * K + j) * 32 + l]; }
    __device__ __forceinline__ int& cnt(int c, int l) { return n[c * 32 + l]; }
    __device__ __forceinline__ void push(int queue, int l, int s) {
        const int j = atomicAdd(&cnt(queue, l), 1);
        slot(queue, j, l) = s;
    }
    __device__ __forceinline__ void bind(Lane<NM, false, false>& L, int s, int l) {
        L.coef = cf + s * 32 + l;
        L.stride = K * 32;
    }
    __device__ __forceinline__ void load(Lane<NM, false, false>& L, int s, int l) {
        L.px = fl(PF_PX, s, l); L.py = fl(PF_PY, s, l); L.pz = fl(PF_PZ, s, l);
        L.dx = fl(PF_DX, s, l); L.dy = fl(PF_DY, s, l); L.dz = fl(PF_DZ, s, l);
        L.e = fl(PF_E, s, l); L.mumax = fl(PF_MUMAX, s, l); L.inv_mumax = fl(PF_INVMU, s, l);
        L.tg = fl(PF_TG, s, l);
        const uint32_t st = u(PF_STATE, s, l);
        L.state = (int)(st & 0xffu);
        L.scattered = (int)(st >> 8);
        L.job = (int)u(PF_JOB, s, l);
        L.nsteps = u(PF_NSTEPS, s, l);
        L.ngath = u(PF_NGATH, s, l);
        L.rs.angle = u(PF_ANGLE, s, l); L.rs.hlo = u(PF_HLO, s, l); L.rs.hhi = u(PF_HHI, s, l);
        L.rs.blk = u(PF_BLK, s, l);
        bind(L, s, l);
    }
    __device__ __forceinline__ void store(const Lane<NM, false, false>& L, int s, int l) {
        fl(PF_PX, s, l) = L.px; fl(PF_PY, s, l) = L.py; fl(PF_PZ, s, l) = L.pz;
        fl(PF_DX, s, l) = L.dx; fl(PF_DY, s, l) = L.dy; fl(PF_DZ, s, l) = L.dz;
        fl(PF_E, s, l) = L.e; fl(PF_MUMAX, s, l) = L.mumax; fl(PF_INVMU, s, l) = L.inv_mumax;
        fl(PF_TG, s, l) = L.tg;
        u(PF_STATE, s, l) = (uint32_t)L.state | ((uint32_t)L.scattered << 8);
        u(PF_JOB, s, l) = (uint32_t)L.job;
        u(PF_NSTEPS, s, l) = L.nsteps;
        u(PF_NGATH, s, l) = L.ngath;
        u(PF_ANGLE, s, l) = L.rs.angle; u(PF_HLO, s, l) = L.rs.hlo; u(PF_HHI, s, l) = L.rs.hhi;
        u(PF_BLK, s, l) = L.rs.blk;
    }
    // a flight that ended stores what the flights changed
    __device__ __forceinline__ void store_flight(const Lane<NM, false, false>& L, int s, int l) {
        fl(PF_PX, s, l) = L.px; fl(PF_PY, s, l) = L.py; fl(PF_PZ, s, l) = L.pz;
        fl(PF_TG, s, l) = L.tg;
        u(PF_STATE, s, l) = (uint32_t)L.state | ((uint32_t)L.scattered << 8);
        u(PF_NSTEPS, s, l) = L.nsteps;
        u(PF_BLK, s, l) = L.rs.blk;
    }
};

// tail: once no idle lane of a warp can take another ready photon and fewer
// than `tail` lanes still fly, the warp parks its photons for the next round
// instead of flying on with a thinning warp, but only photons that have
// flown at least `park_min` (>= 1) flights in this phase: every round moves
// every photon on, so the rounds end
// rounds a block may run (a block's rounds number in the thousands for 1e8
// histories); past it the block records a timeout in P.status and stops
constexpr int POOL_MAX_ROUNDS = 1 << 22;

template <int NM>
__global__ void __launch_bounds__(POOL_THREADS, 3) mc_pool_kernel(const McParams P, int K, int tail, uint32_t park_min) {
    extern __shared__ __align__(16) unsigned char pool_smem[];
    __shared__ unsigned long long cnt[GDRR_NSTATS];
    __shared__ int s_done[POOL_WARPS];
    __shared__ int s_exit;
    using L_t = Lane<NM, false, false>;
    Pool<NM> pl;
    pl.K = K;
    pl.fld = reinterpret_cast<uint32_t*>(pool_smem);
    pl.cf = reinterpret_cast<float*>(pl.fld + (size_t)PF_N * K * 32);
    pl.q = reinterpret_cast<int*>(pl.cf + (size_t)3 * NM * K * 32);
    pl.n = pl.q + (size_t)PQ_N * K * 32;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < GDRR_NSTATS; i += blockDim.x) cnt[i] = 0ull;
    for (int i = threadIdx.x; i < PC_N * 32; i += blockDim.x) pl.n[i] = 0;
    if (threadIdx.x < POOL_WARPS) s_done[threadIdx.x] = 0;
    block_sync();
    if (warp == 0) {
        pl.cnt(PQ_F0, lane) = K;                          // every slot starts free
        for (int j = 0; j < K; ++j) pl.slot(PQ_F0, j, lane) = j;
    }
    L_t L;
    L.state = S_DEAD;
    L.defer_e = false;
    L.need_e = false;
    L.c_steps = 0; L.c_virt = 0; L.c_skip = 0;
    unsigned long long pool_next = 0, pool_end = 0;
    bool exhausted = false;
    block_sync();

    for (int round = 0;; ++round) {
        if (round >= POOL_MAX_ROUNDS) {
            if (threadIdx.x == 0 && P.status) atomicOr(P.status, 2);
            break;
        }
        // queues by round parity: this round's FLIGHT runs qFly (filled by
        // the last round and by this START); photons that fly next round go
        // to qNext; START takes the free slots of qF, freed slots go to qFn
        const int c = round & 1;
        const int qFly = c ? PQ_R0 : PQ_R1, qNext = c ? PQ_R1 : PQ_R0;
        const int qF = c ? PQ_F1 : PQ_F0, qFn = c ? PQ_F0 : PQ_F1;

        // ---- START: free slots of this round take new histories ----------
        if (warp == 0) {
            pl.cnt(PQ_E, lane) = 0;                       // consumed by the last ESCAPE
            // between rounds every slot of a class is free or ready to fly
            const bool whole = pl.cnt(qF, lane) + pl.cnt(qFly, lane) == K;
            const unsigned broken = __ballot_sync(FULL, !whole);
            const int nfree = __reduce_add_sync(FULL, (unsigned)pl.cnt(qF, lane));
            int ndone = 0;
            for (int w = 0; w < POOL_WARPS; ++w) ndone += s_done[w];
            if (lane == 0) {
                s_exit = (nfree == 32 * K && ndone == POOL_WARPS) ? 1 : 0;
                if (broken) {                             // a slot went missing: stop, and say so
                    if (P.status) atomicOr(P.status, 4);
                    s_exit = 1;
                }
            }
        }
        block_sync();
        if (s_exit) break;
        {
            const int nf = pl.cnt(qF, lane);
            int j = warp;
            bool need = j < nf;
            int sl = need ? pl.slot(qF, j, lane) : 0;
            while (!exhausted) {
                const unsigned nb = __ballot_sync(FULL, need);
                if (nb == 0u) break;
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
                const unsigned want = (unsigned)__popc(nb);
                const unsigned take = want < avail ? want : avail;
                const unsigned rank = (unsigned)__popc(nb & ((1u << lane) - 1u));
                if (need && rank < take) {
                    pl.bind(L, sl, lane);
                    L.start(P, P.seg0 + pool_next + rank, cnt);
                    if (L.state == S_FLY) {                 // else it missed the box and was tallied: retry
                        pl.store(L, sl, lane);
                        pl.push(qFly, lane, sl);
                        j += POOL_WARPS;
                        need = j < nf;
                        if (need) sl = pl.slot(qF, j, lane);
                    }
                }
                pool_next += take;
            }
            // free slots that got no history stay free for a later round
            for (; need; ) {
                pl.push(qFn, lane, sl);
                j += POOL_WARPS;
                need = j < nf;
                if (need) sl = pl.slot(qF, j, lane);
            }
            if (lane == 0) s_done[warp] = (exhausted && pool_next >= pool_end) ? 1 : 0;
        }
        block_sync();

        // ---- FLIGHT ---------------------------------------------------------
        if (warp == 0) pl.cnt(qF, lane) = 0;             // consumed by START
        {
            const int nR = pl.cnt(qFly, lane);
            bool have = false, drained = false;
            int sl = 0;
            uint32_t flown = 0;                           // flights of the held photon in this phase
            for (;;) {
                if (!have && !drained) {
                    const int pos = atomicAdd(&pl.cnt(PC_HEAD, lane), 1);
                    if (pos < nR) {
                        sl = pl.slot(qFly, pos, lane);
                        pl.load(L, sl, lane);
                        have = true;
                        flown = 0;
                    } else {
                        drained = true;
                    }
                }
                const unsigned act = __ballot_sync(FULL, have);
                const unsigned idle_open = __ballot_sync(FULL, !have && !drained);
                const unsigned fresh = __ballot_sync(FULL, have && flown < park_min);
                if (act == 0u && idle_open == 0u) break;
                if (idle_open == 0u && fresh == 0u && __popc(act) < tail) {
                    if (have) {                           // park for the next round
                        pl.store_flight(L, sl, lane);
                        pl.push(qNext, lane, sl);
                    }
                    break;
                }
                if (have) {
                    L.step(P, cnt);
                    ++flown;
                    if (L.state != S_FLY) {
                        pl.store_flight(L, sl, lane);
                        if (L.state == S_GATHER) pl.push(PQ_G, lane, sl);
                        else if (L.state == S_ESC) pl.push(PQ_E, lane, sl);
                        else pl.push(qFn, lane, sl);        // step limit: the history ended
                        have = false;
                    }
                }
            }
        }
        block_sync();

        // ---- GATHER -----------------------------------------------------------
        if (warp == 0) {
            // a warp that parks can leave ready photons of a class unpopped
            // (its lane of that class still held one): they fly next round
            const int nR = pl.cnt(qFly, lane);
            for (int pos = pl.cnt(PC_HEAD, lane); pos < nR; ++pos) pl.push(qNext, lane, pl.slot(qFly, pos, lane));
            pl.cnt(qFly, lane) = 0;
            pl.cnt(PC_HEAD, lane) = 0;
        }
        {
            const int nG = pl.cnt(PQ_G, lane);
            for (int j = warp; j < nG; j += POOL_WARPS) {
                const int sl = pl.slot(PQ_G, j, lane);
                pl.load(L, sl, lane);
                L.gather(P, cnt);
                if (L.state == S_DEAD) {
                    pl.push(qFn, lane, sl);               // photoelectric absorption
                } else {
                    pl.u(PF_STATE, sl, lane) = (uint32_t)L.state | ((uint32_t)L.scattered << 8);
                    pl.u(PF_NGATH, sl, lane) = L.ngath;
                    pl.push(L.state == S_FLY ? qNext : PQ_I, lane, sl);
                }
            }
        }
        block_sync();

        // ---- INTER ------------------------------------------------------------
        if (warp == 0) pl.cnt(PQ_G, lane) = 0;
        {
            const int nI = pl.cnt(PQ_I, lane);
            for (int j = warp; j < nI; j += POOL_WARPS) {
                const int sl = pl.slot(PQ_I, j, lane);
                pl.load(L, sl, lane);
                L.interact(P, cnt);
                if (L.state == S_DEAD) {
                    pl.push(qFn, lane, sl);               // energy cut-off
                } else {
                    pl.store(L, sl, lane);
                    pl.push(qNext, lane, sl);
                }
            }
        }
        block_sync();

        // ---- ESCAPE -----------------------------------------------------------
        if (warp == 0) pl.cnt(PQ_I, lane) = 0;
        {
            const int nE = pl.cnt(PQ_E, lane);
            for (int j = warp; j < nE; j += POOL_WARPS) {
                const int sl = pl.slot(PQ_E, j, lane);
                pl.load(L, sl, lane);
                L.escape(P, cnt, true);
                pl.push(qFn, lane, sl);
            }
        }
        block_sync();
    }

    atomicAdd(&cnt[GDRR_ST_STEPS], (unsigned long long)L.c_steps);
    atomicAdd(&cnt[GDRR_ST_VIRTUAL], (unsigned long long)L.c_virt);
    atomicAdd(&cnt[GDRR_ST_CELL_SKIPS], (unsigned long long)L.c_skip);
    block_sync();
    for (int i = threadIdx.x; i < GDRR_NSTATS; i += blockDim.x)
        if (cnt[i]) atomicAdd(P.stats + i, cnt[i]);
}

// Gather roofline probe: the transport's trilinear corner gather (same
// layout, same index arithmetic) at pseudo-random cells, with nothing else,
// so the memory system's ceiling for this access pattern can be measured.
__global__ void __launch_bounds__(256) gather_probe_kernel(const McParams P, uint64_t n_cells,
                                                         unsigned int* sink) {
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t nth = (uint64_t)gridDim.x * blockDim.x;
    float acc = 0.0f;
    for (uint64_t i = tid; i < n_cells; i += nth) {
        uint32_t h = (uint32_t)i * 0x9E3779B1u;
        h ^= h >> 15; h *= 0x2C1B3C6Du; h ^= h >> 12; h *= 0x297A2D39u; h ^= h >> 15;
        const uint32_t h2 = h * 0x85EBCA6Bu ^ (h >> 13);
        const uint32_t h3 = h2 * 0xC2B2AE35u ^ (h2 >> 16);
        const float fx = (float)(h & 0xffffu) * (1.0f / 65536.0f) * (float)P.nx - 0.5f;
        const float fy = (float)(h2 & 0xffffu) * (1.0f / 65536.0f) * (float)P.ny - 0.5f;
        const float fz = (float)(h3 & 0xffffu) * (1.0f / 65536.0f) * (float)P.nz - 0.5f;
        const int gx = (int)floorf(fx), gy = (int)floorf(fy), gz = (int)floorf(fz);
        const float tx = fx - (float)gx, ty = fy - (float)gy, tz = fz - (float)gz;
        const int x0 = min(max(gx, 0), P.nx - 1), x1 = min(max(gx + 1, 0), P.nx - 1);
        const int y0 = min(max(gy, 0), P.ny - 1), y1 = min(max(gy + 1, 0), P.ny - 1);
        const int z0 = min(max(gz, 0), P.nz - 1), z1 = min(max(gz + 1, 0), P.nz - 1);
        const float wxy[4] = {(1.0f - tx) * (1.0f - ty), tx * (1.0f - ty), (1.0f - tx) * ty, tx * ty};
        const int bx[2] = {brick_x(x0), brick_x(x1)};
        const int by[2] = {brick_y(y0, P.bsy), brick_y(y1, P.bsy)};
        const int bz[2] = {brick_z(z0, P.bsz), brick_z(z1, P.bsz)};
        const int rows[4] = {by[0] + bz[0], by[1] + bz[0], by[0] + bz[1], by[1] + bz[1]};
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const uint2 vx = __ldg(P.vox + rows[c >> 1] + bx[c & 1]);
            acc = acc + (wxy[c & 3] * ((c >> 2) ? tz : 1.0f - tz)) * __uint_as_float(vx.x) * (float)(vx.y + 1u);
        }
    }
    if (acc == -1.0f) atomicAdd(sink, 1u);   // keeps the loads; never true for densities >= 0
}

__global__ void stream_words_kernel(const RoundKeys rk, uint32_t angle_index, uint64_t hid0, int n_hist,
                                    int n_blocks, uint32_t* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_hist) return;
    Stream rs;
    rs.init(angle_index, hid0 + (uint64_t)i);
    uint32_t* o = out + (size_t)i * 4 * n_blocks;
    for (int b = 0; b < n_blocks; ++b) {
        const uint4 w = rs.block(rk);
        o[4 * b] = w.x; o[4 * b + 1] = w.y; o[4 * b + 2] = w.z; o[4 * b + 3] = w.w;
    }
}

template <int NM>
constexpr size_t smem_bytes(int block) { return (size_t)3 * NM * block * sizeof(float); }

// Per-thread coefficient tables beyond 47 KB per block (8 materials at 512
// threads) need the kernel's dynamic shared-memory cap raised first.
template <int NM, bool REC, bool GEN, bool LM>
cudaError_t allow_smem(int block) {
    const size_t bytes = smem_bytes<NM>(block);
    if (bytes <= 47 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(mc_kernel<NM, REC, GEN, LM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int NM, bool REC, bool GEN, bool LM>
cudaError_t launch_t(const McParams& p, int block, int grid, cudaStream_t s) {
    const cudaError_t e = allow_smem<NM, REC, GEN, LM>(block);
    if (e != cudaSuccess) return e;
    mc_kernel<NM, REC, GEN, LM><<<grid, block, smem_bytes<NM>(block), s>>>(p);
    return cudaGetLastError();
}

template <int NM, bool REC, bool GEN, bool LM>
int occupancy_t(int block) {
    int n = 0;
    if (allow_smem<NM, REC, GEN, LM>(block) != cudaSuccess
        || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, mc_kernel<NM, REC, GEN, LM>, block, smem_bytes<NM>(block))
               != cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

template <bool REC, bool GEN, bool LM>
cudaError_t launch_nm(const McParams& p, int block, int grid, cudaStream_t s) {
    if (p.n_mat <= 2) return launch_t<2, REC, GEN, LM>(p, block, grid, s);
    if (p.n_mat <= 4) return launch_t<4, REC, GEN, LM>(p, block, grid, s);
    return launch_t<8, REC, GEN, LM>(p, block, grid, s);
}

template <bool REC, bool LM>
int occupancy_nm(int n_mat, int block) {
    if (n_mat <= 2) return occupancy_t<2, REC, false, LM>(block);
    if (n_mat <= 4) return occupancy_t<4, REC, false, LM>(block);
    return occupancy_t<8, REC, false, LM>(block);
}

template <bool LM>
cudaError_t launch_lm(const McParams& p, int block, int grid, bool records, cudaStream_t s) {
    const bool gen = p.nearest_voxel != 0 || p.scatter_filter != 0 || p.ray_ff != 0;
    if (records) return gen ? launch_nm<true, true, LM>(p, block, grid, s) : launch_nm<true, false, LM>(p, block, grid, s);
    return gen ? launch_nm<false, true, LM>(p, block, grid, s) : launch_nm<false, false, LM>(p, block, grid, s);
}

template <int NM>
cudaError_t launch_pool_t(const McParams& p, int K, int grid, cudaStream_t s) {
    const size_t bytes = pool_smem_bytes<NM>(K);
    cudaError_t e = cudaFuncSetAttribute(mc_pool_kernel<NM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    // measured on the 2 mm torso (2 photons per thread): tail 24 / park 4
    // 112.6 ms, tail 16 / park 16 117.1 ms, tail 8 130 ms
    const int tail = p.pool_tail > 0 ? p.pool_tail : 24;
    const uint32_t park_min = p.pool_park_min > 0 ? (uint32_t)p.pool_park_min : 4u;
    mc_pool_kernel<NM><<<grid, POOL_THREADS, bytes, s>>>(p, K, tail, park_min);
    return cudaGetLastError();
}

template <int NM>
int pool_occupancy_t(int K) {
    const size_t bytes = pool_smem_bytes<NM>(K);
    int n = 0;
    if (cudaFuncSetAttribute(mc_pool_kernel<NM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess
        || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, mc_pool_kernel<NM>, POOL_THREADS, bytes) != cudaSuccess)
        return 0;
    return n;
}

}  // namespace

int pool_threads() { return POOL_THREADS; }

// slots per lane class for pool photons per thread
static int pool_k(int per_thread) { return POOL_WARPS * per_thread; }

cudaError_t launch_mc_pool(const McParams& p, int per_thread, int grid, cudaStream_t s) {
    const int K = pool_k(per_thread);
    if (p.n_mat <= 2) return launch_pool_t<2>(p, K, grid, s);
    if (p.n_mat <= 4) return launch_pool_t<4>(p, K, grid, s);
    return launch_pool_t<8>(p, K, grid, s);
}

int mc_pool_occupancy_blocks(int n_mat, int per_thread) {
    const int K = pool_k(per_thread);
    if (n_mat <= 2) return pool_occupancy_t<2>(K);
    if (n_mat <= 4) return pool_occupancy_t<4>(K);
    return pool_occupancy_t<8>(K);
}

cudaError_t launch_mc_source(const McParams& p, cudaStream_t s) {
    if (!p.src || p.total == 0) return cudaErrorInvalidValue;
    int dev = 0, n_sm = 1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const uint64_t blocks = (p.total + 255) / 256;
    const uint64_t cap = (uint64_t)n_sm * 8;
    const int grid = (int)(blocks < cap ? blocks : cap);
    float4* out = const_cast<float4*>(p.src);
    if (p.n_mat <= 2) mc_source_kernel<2><<<grid, 256, 0, s>>>(p, out);
    else if (p.n_mat <= 4) mc_source_kernel<4><<<grid, 256, 0, s>>>(p, out);
    else mc_source_kernel<8><<<grid, 256, 0, s>>>(p, out);
    return cudaGetLastError();
}

cudaError_t launch_mc(const McParams& p, int block, int grid, bool records, cudaStream_t s) {
    if (p.lm) {
        if (!p.cells) return cudaErrorInvalidValue;       // the local majorants are the cell bounds
        return launch_lm<true>(p, block, grid, records, s);
    }
    return launch_lm<false>(p, block, grid, records, s);
}

int mc_occupancy_blocks(int n_mat, int block, bool records, bool lm) {
    if (lm) return records ? occupancy_nm<true, true>(n_mat, block) : occupancy_nm<false, true>(n_mat, block);
    return records ? occupancy_nm<true, false>(n_mat, block) : occupancy_nm<false, false>(n_mat, block);
}

cudaError_t launch_gather_probe(const McParams& p, uint64_t n_cells, int grid, unsigned int* sink, cudaStream_t s) {
    gather_probe_kernel<<<grid, 256, 0, s>>>(p, n_cells, sink);
    return cudaGetLastError();
}

cudaError_t launch_stream_words(uint64_t seed, uint32_t angle_index, uint64_t hid0, int n_hist, int n_blocks,
                                uint32_t* out, cudaStream_t s) {
    if (n_hist <= 0) return cudaSuccess;
    stream_words_kernel<<<(n_hist + 127) / 128, 128, 0, s>>>(round_keys(seed), angle_index, hid0, n_hist, n_blocks,
                                                             out);
    return cudaGetLastError();
}

}  // namespace gdrr
