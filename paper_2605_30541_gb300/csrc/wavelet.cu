// Band-passed Ricker source wavelet of the paper's production runs (Sec.
// "Source Wavelet", Tab. bands): a Ricker pulse of peak frequency f0 centred
// at t0 = 1/f0, filtered by a Butterworth band-pass at [f_lo, f_hi] forward
// and then backward in time (zero phase), divided by its l2 norm and
// multiplied by sqrt((f_hi - f_lo) / 24 Hz).
//
// The filter is designed on the host from the Butterworth definition:
// analog low-pass prototype poles exp(i pi (2k + N + 1) / (2N)), the
// low-pass to band-pass map around w0 = sqrt(w_lo w_hi) with bandwidth
// w_hi - w_lo (edges prewarped, w = 2 fs tan(pi f / fs)), then the bilinear
// map z = (2 fs + s) / (2 fs - s), grouped into second-order sections (each
// a conjugate pole pair with two zeros; gain on the first section).
// Forward-backward filtering follows the usual zero-phase recipe: the signal
// is extended at both ends by its odd reflection about the end samples
// (3 (2 S + 1) samples for S sections, fewer zero coefficients aside; the
// record must be longer than that), each
// pass starts every section in the steady state of a constant input equal to
// the first sample it sees, and the extension is dropped at the end. One
// GPU thread runs the recursion in FP64 (the record is a few thousand
// samples); the result is written in the requested precision.
#include <cmath>
#include <complex>
#include <vector>

#include "sim_internal.h"

namespace gsim {
namespace {

using cd = std::complex<double>;

struct Sos {
    double b0, b1, b2, a1, a2;  // a0 = 1
};

// Digital Butterworth band-pass of order N (2N poles) at [f_lo, f_hi], fs = 1/dt.
std::vector<Sos> butter_bandpass(int N, double f_lo, double f_hi, double fs) {
    const double pi = 3.14159265358979323846;
    const double wl = 2.0 * fs * std::tan(pi * f_lo / fs), wh = 2.0 * fs * std::tan(pi * f_hi / fs);
    const double bw = wh - wl, w0 = std::sqrt(wl * wh);
    std::vector<cd> poles;  // analog band-pass poles
    for (int k = 0; k < N; k++) {
        const cd p = std::exp(cd(0.0, pi * (2.0 * k + N + 1) / (2.0 * N)));  // left half plane, |p| = 1
        const cd a = p * (bw / 2.0), r = std::sqrt(a * a - w0 * w0);
        poles.push_back(a + r);
        poles.push_back(a - r);
    }
    // analog gain bw^N (N zeros at s = 0); bilinear map
    cd gain(std::pow(bw, N), 0.0);
    std::vector<cd> zp;
    for (const cd &p : poles) {
        zp.push_back((2.0 * fs + p) / (2.0 * fs - p));
        gain /= (2.0 * fs - p);
    }
    gain *= std::pow(2.0 * fs, N);  // prod over the N finite zeros (s = 0) of (2 fs - 0)
    // zeros: N at z = 1 (from s = 0), N at z = -1 (from s = infinity)
    // sections: conjugate pairs of poles (upper half plane ones), zeros (1, -1) each
    std::vector<cd> up;
    for (const cd &z : zp)
        if (z.imag() > 0) up.push_back(z);
    std::vector<Sos> s;
    for (size_t i = 0; i < up.size(); i++) {
        Sos q{};
        q.b0 = 1.0;
        q.b1 = 0.0;  // (z - 1)(z + 1) = z^2 - 1
        q.b2 = -1.0;
        q.a1 = -2.0 * up[i].real();
        q.a2 = std::norm(up[i]);
        s.push_back(q);
    }
    if (s.empty()) return s;
    const double g = gain.real();
    s[0].b0 *= g;
    s[0].b1 *= g;
    s[0].b2 *= g;
    return s;
}

// Steady state (transposed direct form II) of each section under a unit
// constant input to the cascade.
std::vector<double> sos_steady(const std::vector<Sos> &s) {
    std::vector<double> zi;
    double scale = 1.0;  // DC gain of the sections before
    for (const Sos &q : s) {
        // y = b0 x + z1, z1' = b1 x - a1 y + z2, z2' = b2 x - a2 y; x = 1 constant, y = dc
        const double dc = (q.b0 + q.b1 + q.b2) / (1.0 + q.a1 + q.a2);
        const double z2 = q.b2 - q.a2 * dc, z1 = q.b1 - q.a1 * dc + z2;
        zi.push_back(scale * z1);
        zi.push_back(scale * z2);
        scale *= dc;
    }
    return zi;
}

constexpr int kMaxSections = 16;
struct Filt {
    int nsec;
    double b0[kMaxSections], b1[kMaxSections], b2[kMaxSections], a1[kMaxSections], a2[kMaxSections];
    double z1[kMaxSections], z2[kMaxSections];  // steady state for a unit input
};

__device__ double ricker_at(double f0, double t) {
    const double pi = 3.14159265358979323846;
    const double a = (pi * f0 * t) * (pi * f0 * t);
    return (1.0 - 2.0 * a) * exp(-a);
}

// one pass of the cascade over x[0..n) in place, started in the steady state of x[0]
__device__ void cascade(const Filt &F, double *x, long long n, int dir) {
    double z1[kMaxSections], z2[kMaxSections];
    const double x0 = dir > 0 ? x[0] : x[n - 1];
    for (int k = 0; k < F.nsec; k++) {
        z1[k] = F.z1[k] * x0;
        z2[k] = F.z2[k] * x0;
    }
    for (long long i = 0; i < n; i++) {
        const long long j = dir > 0 ? i : n - 1 - i;
        double v = x[j];
        for (int k = 0; k < F.nsec; k++) {
            const double y = F.b0[k] * v + z1[k];
            z1[k] = F.b1[k] * v - F.a1[k] * y + z2[k];
            z2[k] = F.b2[k] * v - F.a2[k] * y;
            v = y;
        }
        x[j] = v;
    }
}

__global__ void k_bandpass_ricker(const Filt F, int nt, double dt, double f0, int pad, double scale, double *work,
                                  void *out, int fp64) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    const long long n = nt + 2LL * pad;
    for (int i = 0; i < nt; i++) work[pad + i] = ricker_at(f0, i * dt - 1.0 / f0);
    const double first = work[pad], last = work[pad + nt - 1];
    for (int i = 1; i <= pad; i++) {  // odd reflections about the end samples
        work[pad - i] = 2.0 * first - work[pad + i];
        work[pad + nt - 1 + i] = 2.0 * last - work[pad + nt - 1 - i];
    }
    cascade(F, work, n, +1);
    cascade(F, work, n, -1);
    double ss = 0.0;
    for (int i = 0; i < nt; i++) ss += work[pad + i] * work[pad + i];
    const double c = ss > 0.0 ? scale / sqrt(ss) : 0.0;
    for (int i = 0; i < nt; i++) {
        const double v = c * work[pad + i];
        if (fp64) static_cast<double *>(out)[i] = v;
        else static_cast<float *>(out)[i] = (float)v;
    }
}

}  // namespace
}  // namespace gsim

extern "C" sim_status sim_wavelet_bandpass(int nt, double dt, double f0, double f_lo, double f_hi, int order,
                                           int precision, void *out, void *stream) {
    using namespace gsim;
    if (nt < 2 || !(dt > 0) || !(f0 > 0) || !out || order < 1 || order > kMaxSections ||
        !(f_lo > 0) || !(f_hi > f_lo) || !(f_hi < 0.5 / dt) || (precision != SIM_FP32 && precision != SIM_FP64)) {
        set_thread_error("sim_wavelet_bandpass: need nt >= 2, dt > 0, f0 > 0, 0 < f_lo < f_hi < 1/(2 dt), "
                         "1 <= order <= 16, a known precision and an output array");
        return SIM_ERR_ARG;
    }
    const std::vector<Sos> s = butter_bandpass(order, f_lo, f_hi, 1.0 / dt);
    if ((int)s.size() != order) {
        set_thread_error("sim_wavelet_bandpass: the band-pass has real poles (band too wide for this design)");
        return SIM_ERR_ARG;
    }
    const std::vector<double> zi = sos_steady(s);
    Filt F{};
    F.nsec = (int)s.size();
    for (int k = 0; k < F.nsec; k++) {
        F.b0[k] = s[k].b0;
        F.b1[k] = s[k].b1;
        F.b2[k] = s[k].b2;
        F.a1[k] = s[k].a1;
        F.a2[k] = s[k].a2;
        F.z1[k] = zi[2 * k];
        F.z2[k] = zi[2 * k + 1];
    }
    // extension length: 3 (2 S + 1) less the sections with a zero last
    // coefficient in both numerator and denominator, capped by the record
    int zb = 0, za = 0;
    for (const Sos &q : s) {
        zb += q.b2 == 0.0;
        za += q.a2 == 0.0;
    }
    const int pad = 3 * (2 * F.nsec + 1 - std::min(zb, za));
    if (nt <= pad) {
        set_thread_error("sim_wavelet_bandpass: the record must be longer than the reflection at its ends");
        return SIM_ERR_ARG;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaPointerAttributes attr{};
    const bool dev_out = cudaPointerGetAttributes(&attr, out) == cudaSuccess && attr.type == cudaMemoryTypeDevice;
    cudaGetLastError();
    const size_t esz = precision == SIM_FP64 ? 8 : 4;
    double *work = nullptr;
    void *dout = out;
    cudaError_t e = cudaMalloc(&work, sizeof(double) * (nt + 2 * (size_t)pad));
    if (e == cudaSuccess && !dev_out) e = cudaMalloc(&dout, esz * nt);
    if (e == cudaSuccess) {
        k_bandpass_ricker<<<1, 1, 0, st>>>(F, nt, dt, f0, pad, std::sqrt((f_hi - f_lo) / 24.0), work, dout,
                                           precision == SIM_FP64);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && !dev_out) e = cudaMemcpyAsync(out, dout, esz * nt, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (work) cudaFree(work);
    if (!dev_out && dout) cudaFree(dout);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_thread_error(cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? SIM_ERR_OOM : SIM_ERR_CUDA;
    }
    return SIM_OK;
}
