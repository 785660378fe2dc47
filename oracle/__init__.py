"""CPU oracle of the contour-integral Helmholtz solver (test infrastructure only)."""
