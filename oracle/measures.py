"""Registration performance measures on label maps (oracle; test infrastructure only).

The paper evaluates a registration by transporting the template's label map with the computed
velocity and comparing it with the reference label map (Sec. 5, validation on label maps; the
measures table of App. F):
  * the label map is smoothed with a Gaussian of standard deviation 3 h_x (to avoid Gibbs
    oscillations of the pseudospectral transport), transported with the state equation,
    Eq. (e:state-eq-elim), and thresholded at 0.5;
  * JSC = #(L_R and L_T) / #(L_R or L_T), DSC = 2 #(L_R and L_T) / (#L_R + #L_T),
    FPE = #(L_T minus L_R) / #L_T, FNE = #(L_R minus L_T) / #L_R, with L_T the transported
    template labels and L_R the reference labels.
Reading: the paper transports the labels on a 4x finer grid and injects the result back; here
the transport runs on the problem's own grid (the finer grid only reduces the smoothing and
interpolation error of its real-image data).
"""
import numpy as np

from .fft import fft2, ifft2
from .spectral import spacing, symbols
from .transport import state_solve


def gaussian_smooth(f, sigma):
    """Spectral Gaussian filter with standard deviation sigma (domain units): symbol
    exp(-sigma^2 |k|^2 / 2) with the full |k|^2 (even symbol)."""
    n1, n2 = f.shape
    _, _, KK = symbols(n1, n2)
    return np.real(ifft2(np.exp(-0.5 * sigma * sigma * KK) * fft2(f)))


def overlap(LT, LR):
    """(JSC, DSC, FPE, FNE) of boolean label maps LT (transported template) and LR (reference)."""
    LT = np.asarray(LT, dtype=bool)
    LR = np.asarray(LR, dtype=bool)
    inter = np.count_nonzero(LT & LR)
    union = np.count_nonzero(LT | LR)
    nT, nR = np.count_nonzero(LT), np.count_nonzero(LR)
    jsc = inter / union if union else 1.0
    dsc = 2.0 * inter / (nT + nR) if nT + nR else 1.0
    fpe = np.count_nonzero(LT & ~LR) / nT if nT else 0.0
    fne = np.count_nonzero(LR & ~LT) / nR if nR else 0.0
    return jsc, dsc, fpe, fne


def transported_labels(labels_T, v, nt):
    """Smooth (sigma = 3 h_x), transport with v over nt Heun steps, threshold at 0.5."""
    h1, _ = spacing(labels_T.shape)
    sm = gaussian_smooth(np.asarray(labels_T, dtype=np.float64), 3.0 * h1)
    m1 = state_solve(sm, v, nt)[-1]
    return m1, m1 > 0.5


def label_overlap(labels_T, labels_R, v, nt):
    """The four overlap measures after transporting the template labels with v."""
    _, LT = transported_labels(labels_T, v, nt)
    return overlap(LT, np.asarray(labels_R) > 0.5)
