"""The paper's multi-threaded CPU method (OpenMP), a context implementation timed on the host's cores."""
