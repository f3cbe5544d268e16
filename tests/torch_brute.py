"""An independent float64 PyTorch brute-force renderer for tiny scenes, used to pin the C
oracle (forward and gradients). It shares nothing with the oracle but the conventions:

  * J_phi is not written out: it is torch.autograd's Jacobian of the projection phi, taken
    with create_graph=True so the backward also differentiates J. phi is the equidistant
    model of Sec. 3.2 or, by the camera's `model`, r_d = f r(theta) with r = 2 sin(theta/2),
    2 tan(theta/2), sin(theta) or tan(theta) (pinhole), or the panorama's longitude / latitude
    map (Sec. 6), each written from its definition;
  * R comes from rotating the basis vectors by the quaternion (Hamilton product q v q*);
  * the real spherical harmonics come from the associated-Legendre three-term recursion and
    cos / sin of the azimuth;
  * Sigma_p^-1 is torch.linalg.inv;
  * each pixel's list is sorted by (depth, index) and blended by the rule of Sec. 3.1
    "Rendering" with alpha >= 1/255 kept and the stop before T < 1e-4.
Decisions (visibility, alpha >= 1/255, the stop) are taken on the float64 values.
"""
import math

import torch


def _qmul(a, b):
    aw, ax, ay, az = a.unbind(-1)
    bw, bx, by, bz = b.unbind(-1)
    return torch.stack([aw * bw - ax * bx - ay * by - az * bz,
                        aw * bx + ax * bw + ay * bz - az * by,
                        aw * by - ax * bz + ay * bw + az * bx,
                        aw * bz + ax * by - ay * bx + az * bw], -1)


def _rot_from_quat(q):
    qn = q / q.norm()
    conj = qn * torch.tensor([1.0, -1.0, -1.0, -1.0], dtype=q.dtype)
    cols = []
    for k in range(3):
        v = torch.zeros(4, dtype=q.dtype)
        v[k + 1] = 1.0
        cols.append(_qmul(_qmul(qn, v), conj)[1:])
    return torch.stack(cols, 1)  # columns = rotated basis vectors


def _assoc_legendre(l, m, x):
    """P_l^m(x) with the Condon-Shortley phase, by the standard recursion in l."""
    pmm = torch.ones_like(x)
    if m > 0:
        s = torch.sqrt(torch.clamp(1 - x * x, min=0.0))
        fact = 1.0
        for _ in range(m):
            pmm = -pmm * fact * s
            fact += 2.0
    if l == m:
        return pmm
    pm1 = x * (2 * m + 1) * pmm
    if l == m + 1:
        return pm1
    for ll in range(m + 2, l + 1):
        p = ((2 * ll - 1) * x * pm1 - (ll + m - 1) * pmm) / (ll - m)
        pmm, pm1 = pm1, p
    return pm1


def _real_sh(degree, d):
    ct = d[2]
    phi = torch.atan2(d[1], d[0])
    out = []
    for l in range(degree + 1):
        for m in range(-l, l + 1):
            am = abs(m)
            K = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - am) / math.factorial(l + am))
            P = _assoc_legendre(l, am, ct)
            if m == 0:
                out.append(K * P)
            elif m > 0:
                out.append(math.sqrt(2) * K * P * torch.cos(m * phi))
            else:
                out.append(math.sqrt(2) * K * P * torch.sin(am * phi))
    return torch.stack(out)


def render_and_grad(scene, cam, dLdC=None, bg=(0.0, 0.0, 0.0), grad=True):
    """Returns (image [3,H,W] float64 numpy, dict of gradients or None)."""
    dt = torch.float64
    means = torch.tensor(scene["means"], dtype=dt, requires_grad=grad)
    scales = torch.tensor(scene["scales"], dtype=dt, requires_grad=grad)
    quats = torch.tensor(scene["quats"], dtype=dt, requires_grad=grad)
    opac = torch.tensor(scene["opacities"], dtype=dt, requires_grad=grad)
    sh = torch.tensor(scene["sh"], dtype=dt, requires_grad=grad)
    deg = int(scene["sh_degree"])
    W = torch.tensor(cam["W"], dtype=dt).reshape(3, 3)
    b = torch.tensor(cam["b"], dtype=dt)
    fx, fy, cx, cy = (float(cam[k]) for k in ("fx", "fy", "cx", "cy"))
    w, h = int(cam["width"]), int(cam["height"])
    centre = -(W.T @ b)

    model = int(cam.get("model", 0))
    radial = {0: lambda t: t, 1: lambda t: 2 * torch.sin(t / 2), 2: lambda t: 2 * torch.tan(t / 2),
              3: torch.sin, 5: torch.tan}

    def phi(p):
        if model == 4:
            return torch.stack([cx + fx * torch.atan2(p[0], p[2]),
                                cy + fy * torch.atan2(p[1], torch.sqrt(p[0] ** 2 + p[2] ** 2))])
        lz = torch.sqrt(p[0] ** 2 + p[1] ** 2)
        th = torch.atan2(lz, p[2])
        r = radial[model](th)
        return torch.stack([cx + fx * r * p[0] / lz, cy + fy * r * p[1] / lz])

    def in_field(p):
        if model == 4:
            return float(torch.atan2(p[1].abs(), torch.sqrt(p[0] ** 2 + p[2] ** 2))) < math.pi / 2 - 0.05
        theta = float(torch.atan2(torch.linalg.norm(p[:2]), p[2]))
        return theta < (math.pi / 2 - 0.05 if model in (3, 5) else math.pi - 0.05)

    gs = []
    for i in range(means.shape[0]):
        muc = W @ means[i] + b
        dist = torch.linalg.norm(muc)
        if not (float(dist) > 0.2 and in_field(muc) and float(opac[i]) >= 1 / 255):
            continue
        xy = phi(muc)
        # the pinhole renderer's guard band 1.3 tan(FOV/2), as a cull of the projected mean
        if model == 5 and (abs(float(xy[0]) - cx) > 0.65 * w or abs(float(xy[1]) - cy) > 0.65 * h):
            continue
        J = torch.autograd.functional.jacobian(phi, muc, create_graph=True)
        R = _rot_from_quat(quats[i])
        M = R * scales[i][None, :]
        Sig = M @ M.T
        T = J @ W
        Sp = T @ Sig @ T.T + 0.3 * torch.eye(2, dtype=dt)
        conic = torch.linalg.inv(Sp)
        d = means[i] - centre
        d = d / torch.linalg.norm(d)
        Y = _real_sh(deg, d)
        rgb = torch.clamp(torch.einsum("k,kc->c", Y, sh[i]) + 0.5, min=0.0)
        gs.append((i, float(dist), xy, conic, opac[i], rgb))

    img = torch.zeros(3, h, w, dtype=dt)
    cols = []
    for j in range(h):
        for ii in range(w):
            p = torch.tensor([ii + 0.5, j + 0.5], dtype=dt)
            cand = []
            for (i, dep, xy, conic, o, rgb) in gs:
                dlt = p - xy
                a = torch.clamp(o * torch.exp(-0.5 * dlt @ conic @ dlt), max=0.99)
                if float(a) >= 1 / 255:
                    cand.append((dep, i, a, rgb))
            cand.sort(key=lambda e: (e[0], e[1]))
            T = torch.ones((), dtype=dt)
            C = torch.zeros(3, dtype=dt)
            for (_, _, a, rgb) in cand:
                Tn = T * (1 - a)
                if float(Tn) < 1e-4:
                    break
                C = C + rgb * a * T
                T = Tn
            C = C + T * torch.tensor(bg, dtype=dt)
            cols.append(C)
    img = torch.stack(cols).reshape(h, w, 3).permute(2, 0, 1)
    if not grad:
        return img.detach().numpy(), None
    G = torch.tensor(dLdC, dtype=dt).reshape(3, h, w)
    L = (img * G).sum()
    L.backward()
    z = lambda t: (t.grad if t.grad is not None else torch.zeros_like(t)).numpy()
    return img.detach().numpy(), dict(means=z(means), scales=z(scales), quats=z(quats),
                                      opacities=z(opac), sh=z(sh))
