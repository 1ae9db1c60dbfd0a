// Serving core.
