// Host side: a frame's LOD inputs from a camera (the paper leaves the LOD
// criterion to the application, Sec. 3.3 kernel 4; this library's reading
// is described at cbt_update in cbt.h). Every step is one FP64 operation in
// the order written (built without contraction), then one rounding to FP32,
// so that the same camera gives the same bits wherever it is derived in
// this order.
#include <cmath>

#include "cbt.h"

namespace {

double norm3(const double v[3]) { return std::sqrt((v[0] * v[0] + v[1] * v[1]) + v[2] * v[2]); }

void cross3(const double a[3], const double b[3], double out[3]) {
    out[0] = a[1] * b[2] - a[2] * b[1];
    out[1] = a[2] * b[0] - a[0] * b[2];
    out[2] = a[0] * b[1] - a[1] * b[0];
}

}  // namespace

extern "C" int cbt_frame_from_camera(const cbt_camera* cam, float tau_px, int frustum, cbt_frame* frame) {
    if (!cam || !frame || !(tau_px > 0.0f) || !std::isfinite(tau_px)) return CBT_EINVAL;
    if (!(cam->fovy_rad > 0.0 && cam->fovy_rad < 3.141592653589793) || !(cam->aspect > 0.0) ||
        !std::isfinite(cam->aspect) || cam->height_px <= 0 || cam->width_px <= 0)
        return CBT_EINVAL;
    double f[3], up[3];
    for (int c = 0; c < 3; ++c) {
        f[c] = cam->target[c] - cam->eye[c];
        up[c] = cam->up[c];
        if (!std::isfinite(cam->eye[c]) || !std::isfinite(cam->target[c]) || !std::isfinite(up[c])) return CBT_EINVAL;
    }
    const double fn = norm3(f), un = norm3(up);
    if (!(fn > 0.0) || !(un > 0.0)) return CBT_EINVAL;
    for (int c = 0; c < 3; ++c) f[c] = f[c] / fn;
    // forward, right and up: the up direction falls back to +y (or +x when
    // the view runs along y) when it is nearly parallel to the view
    const double d = (f[0] * (up[0] / un) + f[1] * (up[1] / un)) + f[2] * (up[2] / un);
    double u0[3] = {up[0], up[1], up[2]};
    if (std::fabs(d) > 0.999) {
        const bool along_y = !(std::fabs(f[1]) < 0.9);
        u0[0] = along_y ? 1.0 : 0.0;
        u0[1] = along_y ? 0.0 : 1.0;
        u0[2] = 0.0;
    }
    double r[3], u[3];
    cross3(f, u0, r);
    const double rn = norm3(r);
    if (!(rn > 0.0)) return CBT_EINVAL;
    for (int c = 0; c < 3; ++c) r[c] = r[c] / rn;
    cross3(r, f, u);
    // inward normals of the four side planes and the near plane through the
    // eye; q = (K / tau)^2 with K = height / (2 tan(fovy / 2))
    const double ty = std::tan(cam->fovy_rad / 2.0);
    const double tx = cam->aspect * ty;
    for (int c = 0; c < 3; ++c) {
        frame->planes[0][c] = static_cast<float>(tx * f[c] + r[c]);
        frame->planes[1][c] = static_cast<float>(tx * f[c] - r[c]);
        frame->planes[2][c] = static_cast<float>(ty * f[c] + u[c]);
        frame->planes[3][c] = static_cast<float>(ty * f[c] - u[c]);
        frame->planes[4][c] = static_cast<float>(f[c]);
        frame->eye[c] = cam->eye[c];
    }
    const double K = static_cast<double>(cam->height_px) / (2.0 * ty);
    const double kq = K / static_cast<double>(tau_px);
    frame->q = static_cast<float>(kq * kq);
    frame->nplanes = frustum ? 5u : 0u;
    return CBT_OK;
}
