"""Plain FP64 NumPy statements of the training pieces (test infrastructure, like the rest of
oracle/): the L1 loss and its gradient, and one Adam step (Kingma & Ba, Algorithm 1: biased
moment estimates, bias correction, parameter update) on raw parameters whose activated values
(identity, exp or sigmoid) are what the renderer consumes."""
import numpy as np

ACT_NONE, ACT_EXP, ACT_SIGMOID = 0, 1, 2


def activate(raw, activation):
    raw = np.asarray(raw, np.float64)
    if activation == ACT_EXP:
        return np.exp(raw)
    if activation == ACT_SIGMOID:
        return 1.0 / (1.0 + np.exp(-raw))
    return raw.copy()


def loss_l1(image, target, scale):
    d = np.asarray(image, np.float64) - np.asarray(target, np.float64)
    return scale * np.abs(d).sum(), scale * np.sign(d)


def adam_step(raw, grad_act, m, v, activation, lr, beta1, beta2, eps, t):
    """Returns (raw', act', m', v'). grad_act is dL/d(act(raw)); t >= 1."""
    raw = np.asarray(raw, np.float64)
    a = activate(raw, activation)
    if activation == ACT_EXP:
        g = grad_act * a                  # d exp(r)/dr = exp(r)
    elif activation == ACT_SIGMOID:
        g = grad_act * a * (1.0 - a)      # d s(r)/dr = s (1 - s)
    else:
        g = np.asarray(grad_act, np.float64)
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    raw = raw - lr * mhat / (np.sqrt(vhat) + eps)
    return raw, activate(raw, activation), m, v
