"""Plain CPU oracle of pdGRASS off-tree edge recovery (test infrastructure only)."""
